"""Thin Python binding of libspinmc (include/spinmc.h).

Argument marshalling only: every function below forwards to the C function of
the same name, and every step of a sweep runs in the library's CUDA kernels.
PyTorch supplies device memory and streams (the ``Lattice`` helper allocates
its buffer as a torch uint8 tensor and passes the current CUDA stream).

Importing this module loads ``libspinmc.so`` from the package directory and
raises ImportError if it has not been built (``python -c "import
__graft_entry__ as g; g.build()"``); there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspinmc.so")

SL_OK, SL_EINVAL, SL_ENOMEM, SL_ECUDA, SL_ETIMEOUT, SL_EDEVICE = 0, -1, -2, -3, -4, -5
SL_J_UNIFORM, SL_J_BONDS = 0, 1
SL_STORE_I8, SL_STORE_BITS, SL_STORE_F32_ANGLE, SL_STORE_F32_VEC = 0, 1, 2, 3
SL_OPT_RENORM_EVERY, SL_OPT_FAST_MATH, SL_OPT_KERNEL, SL_OPT_ROWS, SL_OPT_GRAPH = 1, 2, 3, 4, 5
SL_OPT_UPDATE, SL_OPT_MULTIHIT, SL_OPT_TILE, SL_OPT_BLOCKS_PER_SM = 6, 7, 8, 9
SL_UPDATE_METROPOLIS, SL_UPDATE_HEATBATH, SL_UPDATE_SW = 0, 1, 2
SL_WOPT_SPINS_SMEM = 1
SL_BOPT_AUTOTUNE, SL_BOPT_PACK = 1, 2
SL_MB_PHILOX, SL_MB_IMAD, SL_MB_FFMA, SL_MB_MUFU = 0, 1, 2, 3

if not os.path.exists(LIB_PATH):
    raise ImportError("libspinmc.so is not built at %s; run paper_1107_5463_gb300.build.build()"
                      % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

_vp, _int, _u32, _u64, _i64, _dbl, _sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32,
                                          ctypes.c_uint64, ctypes.c_int64, ctypes.c_double,
                                          ctypes.c_size_t)


def _sig(name, restype, *argtypes):
    f = getattr(_lib, name)
    f.restype = restype
    f.argtypes = list(argtypes)
    return f


_sig("sl_required_bytes", _int, _int, _int, _int, _int, _int, ctypes.POINTER(_sz))
_sig("sl_create", _int, _int, _int, _int, _int, _int, _dbl, _vp, _u64, _u32, _vp, _sz, _vp,
     ctypes.POINTER(_vp))
_sig("sl_sweep", _int, _vp, _dbl, _i64, _u64)
_sig("sl_sweep_series", _int, _vp, _dbl, _i64, _u64, _vp, _vp)
_sig("sl_measure", _int, _vp, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl))
_sig("sl_get_spins", _int, _vp, _vp)
_sig("sl_set_spins", _int, _vp, _vp)
_sig("sl_get_state", _int, _vp, ctypes.POINTER(_u64), ctypes.POINTER(_i64))
_sig("sl_set_state", _int, _vp, _i64)
_sig("sl_set_option", _int, _vp, _int, _i64)
_sig("sl_autotune", _int, _vp, _dbl, _int, ctypes.c_char_p, ctypes.POINTER(_int),
     ctypes.POINTER(_int))
_sig("sl_destroy", None, _vp)
_sig("sl_workspace_bytes", _int, _vp, _int, ctypes.POINTER(_sz))
_sig("sl_attach_workspace", _int, _vp, _vp, _sz)
_sig("sl_slab_required_bytes", _int, _int, _int, _int, _int, _int, ctypes.POINTER(_sz))
_sig("sl_slab_create", _int, _int, _int, _int, _dbl, _u64, _u32, _int, _int, _vp, _sz, _vp,
     ctypes.POINTER(_vp))
_sig("sl_slab_planes", _int, _vp, _int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
     ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_sz))
_sig("sl_slab_series", _int, _vp, _vp, _vp)
_sig("sl_slab_pass", _int, _vp, _dbl, _u64, _int)
_sig("sl_slabs_exchange", _int, _vp, _int, _int)
_sig("sl_slabs_sweep", _int, _vp, _int, _dbl, _i64, _u64, _vp)
_sig("sl_series_reduce", _int, _vp, _int, _i64, _dbl, _vp, _vp, _vp)
_sig("sl_batch_required_bytes", _int, _int, _vp, _int, _int, _vp, ctypes.POINTER(_sz))
_sig("sl_batch_create", _int, _int, _vp, _int, _int, _vp, _u64, _u32, _vp, _sz, _vp,
     ctypes.POINTER(_vp))
_sig("sl_batch_run", _int, _vp, _i64, _u64, _vp)
_sig("sl_batch_get", _int, _vp, _int, _int, _vp, ctypes.POINTER(_int))
_sig("sl_batch_get_bonds", _int, _vp, _int, _vp)
_sig("sl_batch_sweeps_done", _int, _vp, ctypes.POINTER(_i64))
_sig("sl_batch_set", _int, _vp, _int, _vp, _vp)
_sig("sl_batch_set_sweeps_done", _int, _vp, _i64)
_sig("sl_batch_destroy", None, _vp)
_sig("sl_batch_set_option", _int, _vp, _int, _i64)
_sig("sl_batch_tuning", _int, _vp, _int, ctypes.POINTER(_int), ctypes.POINTER(_int),
     ctypes.POINTER(_dbl))
_sig("sl_ising_measure_static", _int, _int, _int, _dbl, _vp, _vp, _vp)
_sig("sl_microbench_threads", _int, ctypes.POINTER(_int))
_sig("sl_wait_selftest", _int, _vp, ctypes.POINTER(_int))
_sig("sl_microbench", _int, _int, _int, _vp, _sz, _vp, ctypes.POINTER(_dbl))
_sig("sl_walkers_required_bytes", _int, _int, _int, _vp, _vp, _int, ctypes.POINTER(_sz))
_sig("sl_walkers_create", _int, _int, _int, _vp, _vp, _int, _u64, _vp, _sz, _vp,
     ctypes.POINTER(_vp))
_sig("sl_wl_run", _int, _vp, _i64, _int, _int, _u64)
_sig("sl_muca_run", _int, _vp, _vp, _i64, _u64)
_sig("sl_walkers_read", _int, _vp, _vp, _vp, _vp, _vp, _vp)
_sig("sl_walkers_get_spins", _int, _vp, _int, _vp)
_sig("sl_walkers_set_spins", _int, _vp, _int, _vp)
_sig("sl_walkers_write", _int, _vp, _vp, _vp, _vp, _vp)
_sig("sl_walkers_set_sweeps_done", _int, _vp, _i64)
_sig("sl_walkers_info", _int, _vp, ctypes.POINTER(_int), ctypes.POINTER(_int),
     ctypes.POINTER(_i64))
_sig("sl_walkers_destroy", None, _vp)
_sig("sl_walkers_set_option", _int, _vp, _int, _i64)
_sig("sl_dos_glue", _int, _int, _int, _vp, _vp, _vp, _int, _vp, _vp)
_sig("sl_strerror", ctypes.c_char_p, _int)
_sig("sl_last_error", _int, ctypes.c_char_p, _sz)


class SpinMCError(RuntimeError):
    def __init__(self, status, where):
        buf = ctypes.create_string_buffer(512)
        _lib.sl_last_error(buf, 512)
        super().__init__("%s: %s (%d): %s" % (where, _lib.sl_strerror(status).decode(), status,
                                              buf.value.decode(errors="replace")))
        self.status = status


def _check(status, where):
    if status != SL_OK:
        raise SpinMCError(status, where)
    return status


def _addr(x):
    """Raw address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


# ---------------------------------------------------------- raw C ABI ----

def sl_required_bytes(d, L, n, j_layout, storage):
    out = _sz()
    _check(_lib.sl_required_bytes(d, L, n, j_layout, storage, ctypes.byref(out)),
           "sl_required_bytes")
    return out.value


def sl_create(d, L, n, j_layout, storage, J, J_bonds, seed, replica, dev_buf, dev_buf_bytes,
              stream):
    h = _vp()
    _check(_lib.sl_create(d, L, n, j_layout, storage, J, _addr(J_bonds), seed, replica,
                          _addr(dev_buf), dev_buf_bytes, stream, ctypes.byref(h)), "sl_create")
    return h.value


def sl_sweep(h, beta, nsweeps, seed):
    _check(_lib.sl_sweep(h, beta, nsweeps, seed), "sl_sweep")


def sl_sweep_series(h, beta, nsweeps, seed, dev_E, dev_absm):
    _check(_lib.sl_sweep_series(h, beta, nsweeps, seed, _addr(dev_E), _addr(dev_absm)),
           "sl_sweep_series")


def sl_measure(h, n):
    E = _dbl()
    M = (_dbl * (n + 1))()
    _check(_lib.sl_measure(h, ctypes.byref(E), M), "sl_measure")
    return E.value, np.array(M[:])


def sl_get_spins(h, dst):
    _check(_lib.sl_get_spins(h, _addr(dst)), "sl_get_spins")


def sl_set_spins(h, src):
    _check(_lib.sl_set_spins(h, _addr(src)), "sl_set_spins")


def sl_get_state(h):
    s, t = _u64(), _i64()
    _check(_lib.sl_get_state(h, ctypes.byref(s), ctypes.byref(t)), "sl_get_state")
    return s.value, t.value


def sl_set_state(h, sweeps_done):
    _check(_lib.sl_set_state(h, sweeps_done), "sl_set_state")


def sl_set_option(h, option, value):
    _check(_lib.sl_set_option(h, option, value), "sl_set_option")


def sl_autotune(h, beta, trial_sweeps, cache_path=None):
    """Tune the streaming kernels' launch shape; returns (rows, blocks_per_sm)."""
    r, c = _int(), _int()
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(_lib.sl_autotune(h, beta, trial_sweeps, path, ctypes.byref(r), ctypes.byref(c)),
           "sl_autotune")
    return r.value, c.value


def sl_destroy(h):
    _lib.sl_destroy(h)


def sl_workspace_bytes(h, update):
    out = _sz()
    _check(_lib.sl_workspace_bytes(h, update, ctypes.byref(out)), "sl_workspace_bytes")
    return out.value


def sl_attach_workspace(h, dev_buf, nbytes):
    _check(_lib.sl_attach_workspace(h, _addr(dev_buf), nbytes), "sl_attach_workspace")


def sl_slab_required_bytes(d, L, storage, z0, Lz):
    out = _sz()
    _check(_lib.sl_slab_required_bytes(d, L, storage, z0, Lz, ctypes.byref(out)),
           "sl_slab_required_bytes")
    return out.value


def sl_slab_create(d, L, storage, J, seed, replica, z0, Lz, dev_buf, dev_buf_bytes, stream):
    h = _vp()
    _check(_lib.sl_slab_create(d, L, storage, J, seed, replica, z0, Lz, _addr(dev_buf),
                               dev_buf_bytes, stream, ctypes.byref(h)), "sl_slab_create")
    return h.value


def sl_slab_planes(h, colour):
    """(send_lo, send_hi, recv_lo, recv_hi) device addresses and the plane bytes."""
    p = [_vp() for _ in range(4)]
    nb = _sz()
    _check(_lib.sl_slab_planes(h, colour, *[ctypes.byref(x) for x in p], ctypes.byref(nb)),
           "sl_slab_planes")
    return [x.value for x in p], nb.value


def sl_slab_series(h, dev_E, dev_M):
    _check(_lib.sl_slab_series(h, _addr(dev_E), _addr(dev_M)), "sl_slab_series")


def sl_slab_pass(h, beta, seed, colour):
    _check(_lib.sl_slab_pass(h, beta, seed, colour), "sl_slab_pass")


def _ptr_array(xs):
    arr = (_vp * len(xs))(*[_addr(x) for x in xs])
    return arr


def sl_slabs_exchange(handles, colour):
    _check(_lib.sl_slabs_exchange(_ptr_array(handles), len(handles), colour),
           "sl_slabs_exchange")


def sl_slabs_sweep(handles, beta, nsweeps, seed, parts=None):
    p = None if parts is None else _ptr_array(parts)
    _check(_lib.sl_slabs_sweep(_ptr_array(handles), len(handles), beta, nsweeps, seed, p),
           "sl_slabs_sweep")


def sl_series_reduce(parts, nsweeps, N, dev_E, dev_absm, stream):
    _check(_lib.sl_series_reduce(_ptr_array(parts), len(parts), nsweeps, N, _addr(dev_E),
                                 _addr(dev_absm), stream), "sl_series_reduce")


def _i32_array(xs):
    a = np.ascontiguousarray(xs, np.int32)
    return a, a.ctypes.data


def _f64_array(xs):
    a = np.ascontiguousarray(xs, np.float64)
    return a, a.ctypes.data


def sl_batch_required_bytes(d, L_per_sample, ntemps, betas):
    Ls, pL = _i32_array(L_per_sample)
    bs, pb = _f64_array(betas)
    out = _sz()
    _check(_lib.sl_batch_required_bytes(d, pL, Ls.size, ntemps, pb, ctypes.byref(out)),
           "sl_batch_required_bytes")
    return out.value


def sl_batch_create(d, L_per_sample, ntemps, betas, seed, first_sample, dev_buf, dev_buf_bytes,
                    stream):
    Ls, pL = _i32_array(L_per_sample)
    bs, pb = _f64_array(betas)
    h = _vp()
    _check(_lib.sl_batch_create(d, pL, Ls.size, ntemps, pb, seed, first_sample, _addr(dev_buf),
                                dev_buf_bytes, stream, ctypes.byref(h)), "sl_batch_create")
    return h.value


def sl_batch_run(h, nsweeps, seed, dev_E):
    _check(_lib.sl_batch_run(h, nsweeps, seed, _addr(dev_E)), "sl_batch_run")


def sl_batch_get(h, sample, slot, dst):
    k = _int()
    _check(_lib.sl_batch_get(h, sample, slot, _addr(dst), ctypes.byref(k)), "sl_batch_get")
    return k.value


def sl_batch_get_bonds(h, sample, dst):
    _check(_lib.sl_batch_get_bonds(h, sample, _addr(dst)), "sl_batch_get_bonds")


def sl_batch_sweeps_done(h):
    t = _i64()
    _check(_lib.sl_batch_sweeps_done(h, ctypes.byref(t)), "sl_batch_sweeps_done")
    return t.value


def sl_batch_set(h, sample, spins, slot_of_temp):
    """Load a sample's slots (ntemps x N int8 +-1) and slot-of-temperature map."""
    perm, pp = _i32_array(slot_of_temp)
    _check(_lib.sl_batch_set(h, sample, _addr(spins), pp), "sl_batch_set")


def sl_batch_set_sweeps_done(h, sweeps_done):
    _check(_lib.sl_batch_set_sweeps_done(h, sweeps_done), "sl_batch_set_sweeps_done")


def sl_batch_destroy(h):
    _lib.sl_batch_destroy(h)


def sl_batch_set_option(h, option, value):
    _check(_lib.sl_batch_set_option(h, option, value), "sl_batch_set_option")


def sl_batch_tuning(h):
    """[(L, pack, ms per sample-sweep)] for every size class, largest first."""
    out = []
    cls = 0
    while True:
        L, k, ms = _int(), _int(), _dbl()
        n = _lib.sl_batch_tuning(h, cls, ctypes.byref(L), ctypes.byref(k), ctypes.byref(ms))
        if n < 0:
            if cls == 0:
                _check(n, "sl_batch_tuning")
            break
        out.append((L.value, k.value, ms.value))
        cls += 1
        if cls >= n:
            break
    return out


def sl_wait_selftest(stream):
    """1 if the bounded wait of the staged kernels gave up as designed."""
    r = _int()
    _check(_lib.sl_wait_selftest(stream, ctypes.byref(r)), "sl_wait_selftest")
    return r.value


def sl_microbench_threads():
    n = _int()
    _check(_lib.sl_microbench_threads(ctypes.byref(n)), "sl_microbench_threads")
    return n.value


def sl_microbench(kind, iterations, dev_out, nbytes, stream):
    """Launch one microbenchmark (SL_MB_*) on `stream`; return the operations
    it performs (the caller times it)."""
    ops = _dbl()
    _check(_lib.sl_microbench(kind, iterations, _addr(dev_out), nbytes, stream,
                              ctypes.byref(ops)), "sl_microbench")
    return ops.value


def sl_ising_measure_static(d, L, J, dev_spins, dev_out, stream):
    """Energy and magnetisation of a natural-order int8 configuration on the
    device into dev_out[0:2], with no device allocation (see the header)."""
    _check(_lib.sl_ising_measure_static(d, L, J, _addr(dev_spins), _addr(dev_out), stream),
           "sl_ising_measure_static")


def sl_walkers_required_bytes(L, klo, khi, walkers_per_window):
    lo, plo = _i32_array(klo)
    hi, phi = _i32_array(khi)
    out = _sz()
    _check(_lib.sl_walkers_required_bytes(L, lo.size, plo, phi, walkers_per_window,
                                          ctypes.byref(out)), "sl_walkers_required_bytes")
    return out.value


def sl_walkers_create(L, klo, khi, walkers_per_window, seed, dev_buf, dev_buf_bytes, stream):
    lo, plo = _i32_array(klo)
    hi, phi = _i32_array(khi)
    h = _vp()
    _check(_lib.sl_walkers_create(L, lo.size, plo, phi, walkers_per_window, seed, _addr(dev_buf),
                                  dev_buf_bytes, stream, ctypes.byref(h)), "sl_walkers_create")
    return h.value


def sl_wl_run(h, nsweeps, final_stage, flat_percent, seed):
    _check(_lib.sl_wl_run(h, nsweeps, final_stage, flat_percent, seed), "sl_wl_run")


def sl_muca_run(h, lnW, nsweeps, seed):
    W, pW = _f64_array(lnW)
    _check(_lib.sl_muca_run(h, pW, nsweeps, seed), "sl_muca_run")


def sl_walkers_info(h):
    n, k, t = _int(), _int(), _i64()
    _check(_lib.sl_walkers_info(h, ctypes.byref(n), ctypes.byref(k), ctypes.byref(t)),
           "sl_walkers_info")
    return n.value, k.value, t.value


def sl_walkers_read(h):
    """(S int64 [walker][kmax], H uint32 [walker][kmax], level, stage, visited)."""
    n, k, _ = sl_walkers_info(h)
    S = np.empty((n, k), np.int64)
    H = np.empty((n, k), np.uint32)
    lev = np.empty(n, np.int32)
    st = np.empty(n, np.int32)
    vis = np.empty(n, np.uint64)
    _check(_lib.sl_walkers_read(h, S.ctypes.data, H.ctypes.data, lev.ctypes.data, st.ctypes.data,
                                vis.ctypes.data), "sl_walkers_read")
    return S, H, lev, st, vis


def sl_walkers_get_spins(h, walker, dst):
    _check(_lib.sl_walkers_get_spins(h, walker, _addr(dst)), "sl_walkers_get_spins")


def sl_walkers_set_spins(h, walker, src):
    _check(_lib.sl_walkers_set_spins(h, walker, _addr(src)), "sl_walkers_set_spins")


def sl_walkers_write(h, S=None, H=None, stage=None, visited=None):
    """Set S, H ([walker][kmax]), stages and visited masks (None keeps one)."""
    arrs = []
    for a, dt in ((S, np.int64), (H, np.uint32), (stage, np.int32), (visited, np.uint64)):
        arrs.append(None if a is None else np.ascontiguousarray(a, dt))
    _check(_lib.sl_walkers_write(h, *[None if a is None else a.ctypes.data for a in arrs]),
           "sl_walkers_write")


def sl_walkers_set_sweeps_done(h, sweeps_done):
    _check(_lib.sl_walkers_set_sweeps_done(h, sweeps_done), "sl_walkers_set_sweeps_done")


def sl_walkers_destroy(h):
    _lib.sl_walkers_destroy(h)


def sl_walkers_set_option(h, option, value):
    _check(_lib.sl_walkers_set_option(h, option, value), "sl_walkers_set_option")


def sl_dos_glue(L, klo, khi, S, visited):
    """Glue window estimates S[w, q] (level klo[w] + q) into ln g over 0..N."""
    lo, plo = _i32_array(klo)
    hi, phi = _i32_array(khi)
    S = np.ascontiguousarray(S, np.float64)
    vis = np.ascontiguousarray(visited, np.uint64)
    out = np.empty(L * L + 1)
    _check(_lib.sl_dos_glue(L, lo.size, plo, phi, S.ctypes.data, S.shape[1], vis.ctypes.data,
                            out.ctypes.data), "sl_dos_glue")
    return out


# ------------------------------------------------- torch-backed helper ----

_STORAGE_OF_N = {1: SL_STORE_I8, 2: SL_STORE_F32_ANGLE, 3: SL_STORE_F32_VEC}
_NAT_DTYPE = {1: np.int8, 2: np.float32, 3: np.float32}


class Lattice:
    """A lattice whose device buffer is a torch CUDA tensor.

    Spins exchanged with the host are natural-order numpy arrays: int8 +-1
    (n = 1), float32 angles (n = 2), float32 (N, 3) vectors (n = 3)."""

    def __init__(self, d, L, n=1, J=1.0, J_bonds=None, seed=0, replica=0, storage=None,
                 stream=None, device="cuda"):
        import torch
        self.d, self.L, self.n = d, L, n
        self.N = L ** d
        self.storage = _STORAGE_OF_N[n] if storage is None else storage
        j_layout = SL_J_UNIFORM if J_bonds is None else SL_J_BONDS
        nbytes = sl_required_bytes(d, L, n, j_layout, self.storage)
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = torch.cuda.current_stream(self.buf.device) if stream is None else stream
        if J_bonds is not None and isinstance(J_bonds, np.ndarray):
            J_bonds = np.ascontiguousarray(J_bonds, np.int8 if n == 1 else np.float32)
        self._bonds_keepalive = J_bonds
        self.h = sl_create(d, L, n, j_layout, self.storage, J, J_bonds, seed, replica, self.buf,
                           nbytes, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            sl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, beta, nsweeps, seed):
        sl_sweep(self.h, beta, nsweeps, seed)

    def sweep_series(self, beta, nsweeps, seed):
        """Run sweeps and return (E, |m|) as torch float64 CUDA tensors."""
        import torch
        E = torch.empty(nsweeps, dtype=torch.float64, device=self.buf.device)
        m = torch.empty(nsweeps, dtype=torch.float64, device=self.buf.device)
        sl_sweep_series(self.h, beta, nsweeps, seed, E, m)
        return E, m

    def measure(self):
        return sl_measure(self.h, self.n)

    def get_spins(self):
        shape = (self.N,) if self.n != 3 else (self.N, 3)
        out = np.empty(shape, _NAT_DTYPE[self.n])
        sl_get_spins(self.h, out)
        return out

    def set_spins(self, s):
        s = np.ascontiguousarray(s, _NAT_DTYPE[self.n])
        assert s.size == self.N * (3 if self.n == 3 else 1)
        sl_set_spins(self.h, s)

    def state(self):
        return sl_get_state(self.h)

    def set_state(self, sweeps_done):
        sl_set_state(self.h, sweeps_done)

    def set_option(self, option, value):
        sl_set_option(self.h, option, value)

    def autotune(self, beta, trial_sweeps=4, cache_path=None):
        """Pick rows per thread and the grid cap by timing; (rows, blocks_per_sm)."""
        return sl_autotune(self.h, beta, trial_sweeps, cache_path)

    def set_update(self, rule):
        """Select an SL_UPDATE_* rule, attaching a torch-allocated workspace
        first when the rule needs one."""
        import torch
        need = sl_workspace_bytes(self.h, rule)
        if need and (getattr(self, "ws", None) is None or self.ws.numel() < need):
            self.ws = torch.empty(need, dtype=torch.uint8, device=self.buf.device)
            sl_attach_workspace(self.h, self.ws, need)
        sl_set_option(self.h, SL_OPT_UPDATE, rule)


class Slab(Lattice):
    """One slab (planes z0 .. z0 + Lz - 1 along the slowest axis) of an L^d
    Ising lattice, its device buffer a torch CUDA tensor.  The planes of the
    halo exchange are exposed as uint8 tensor views of that buffer."""

    def __init__(self, d, L, z0, Lz, J=1.0, seed=0, replica=0, storage=SL_STORE_I8, stream=None,
                 device="cuda"):
        import torch
        self.d, self.L, self.n = d, L, 1
        self.z0, self.Lz = z0, Lz
        self.N = L ** (d - 1) * Lz
        self.storage = storage
        nbytes = sl_slab_required_bytes(d, L, storage, z0, Lz)
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = torch.cuda.current_stream(self.buf.device) if stream is None else stream
        self._bonds_keepalive = None
        self.h = sl_slab_create(d, L, storage, J, seed, replica, z0, Lz, self.buf, nbytes,
                                self.stream.cuda_stream)

    def planes(self, colour):
        """(send_lo, send_hi, recv_lo, recv_hi) as uint8 views of the buffer."""
        addrs, nb = sl_slab_planes(self.h, colour)
        base = self.buf.data_ptr()
        return [self.buf[a - base:a - base + nb] for a in addrs]

    def series(self, dev_E, dev_M):
        sl_slab_series(self.h, dev_E, dev_M)

    def pass_(self, beta, seed, colour):
        sl_slab_pass(self.h, beta, seed, colour)

    def reduce_series(self, EM, nsweeps, N):
        """(E, |m|) from summed shares (nsweeps energies, then nsweeps M)."""
        import torch
        E = torch.empty(nsweeps, dtype=torch.float64, device=self.buf.device)
        m = torch.empty_like(E)
        sl_series_reduce([EM], nsweeps, N, E, m, self.stream.cuda_stream)
        return E, m


def slabs_sweep(slabs, beta, nsweeps, seed):
    """nsweeps sweeps of in-process slabs (which tile the lattice in order)
    with the library's exchanges; returns (E, |m|) of the whole lattice as
    torch float64 tensors on slab 0's device."""
    import torch
    dev = slabs[0].buf.device
    if any(s.buf.device != dev for s in slabs):
        raise ValueError("slabs_sweep sums the series on one device; call sl_slabs_sweep "
                         "and sl_series_reduce for slabs on several devices")
    parts = [torch.empty(2 * nsweeps, dtype=torch.float64, device=dev) for s in slabs]
    sl_slabs_sweep([s.h for s in slabs], beta, nsweeps, seed, parts)
    E = torch.empty(nsweeps, dtype=torch.float64, device=dev)
    m = torch.empty_like(E)
    N = float(slabs[0].L ** slabs[0].d)
    sl_series_reduce(parts, nsweeps, N, E, m, slabs[0].stream.cuda_stream)
    return E, m


class Walkers:
    """Windowed multicanonical / Wang-Landau walkers, the device buffer a
    torch CUDA tensor."""

    def __init__(self, L, klo, khi, walkers_per_window, seed=0, stream=None, device="cuda"):
        import torch
        self.L = L
        self.N = L * L
        self.klo = np.asarray(klo, np.int32)
        self.khi = np.asarray(khi, np.int32)
        self.wpw = walkers_per_window
        nbytes = sl_walkers_required_bytes(L, self.klo, self.khi, walkers_per_window)
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = torch.cuda.current_stream(self.buf.device) if stream is None else stream
        self.h = sl_walkers_create(L, self.klo, self.khi, walkers_per_window, seed, self.buf,
                                   nbytes, self.stream.cuda_stream)
        self.nwalk, self.kmax, _ = sl_walkers_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            sl_walkers_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option, value):
        sl_walkers_set_option(self.h, option, value)

    def wl(self, nsweeps, final_stage, flat_percent=80, seed=0):
        sl_wl_run(self.h, nsweeps, final_stage, flat_percent, seed)

    def muca(self, lnW, nsweeps, seed=0):
        lnW = np.ascontiguousarray(lnW, np.float64)
        assert lnW.shape == (len(self.klo), self.kmax)
        sl_muca_run(self.h, lnW, nsweeps, seed)

    def read(self):
        return sl_walkers_read(self.h)

    def spins(self, walker):
        out = np.empty(self.N, np.int8)
        sl_walkers_get_spins(self.h, walker, out)
        return out

    def save(self):
        """Checkpoint: (spins [walker][N], S, H, stage, visited, sweeps done)."""
        S, H, _, stage, vis = self.read()
        spins = np.stack([self.spins(j) for j in range(self.nwalk)])
        return spins, S, H, stage, vis, sl_walkers_info(self.h)[2]

    def load(self, ckpt):
        spins, S, H, stage, vis, t = ckpt
        for j in range(self.nwalk):
            sl_walkers_set_spins(self.h, j, np.ascontiguousarray(spins[j], np.int8))
        sl_walkers_write(self.h, S, H, stage, vis)
        sl_walkers_set_sweeps_done(self.h, t)


class Batch:
    """A batch of Edwards-Anderson samples with replica exchange, its device
    buffer a torch CUDA tensor.  L_per_sample[q] is the side of the sample with
    global index first_sample + q."""

    def __init__(self, d, L_per_sample, ntemps, betas, seed=0, first_sample=0, stream=None,
                 device="cuda"):
        import torch
        self.d = d
        self.L = [int(x) for x in L_per_sample]
        self.ntemps = ntemps
        self.nsamples = len(self.L)
        self.first_sample = first_sample
        nbytes = sl_batch_required_bytes(d, self.L, ntemps, betas)
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = torch.cuda.current_stream(self.buf.device) if stream is None else stream
        self.h = sl_batch_create(d, self.L, ntemps, betas, seed, first_sample, self.buf, nbytes,
                                 self.stream.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            sl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, nsweeps, seed, series=False):
        """Run sweeps; with series=True return the energies as a torch float64
        tensor of shape (nsamples, nsweeps, ntemps)."""
        import torch
        E = None
        if series:
            E = torch.empty((self.nsamples, nsweeps, self.ntemps), dtype=torch.float64,
                            device=self.buf.device)
        sl_batch_run(self.h, nsweeps, seed, E)
        return E

    def set_option(self, option, value):
        sl_batch_set_option(self.h, option, value)

    def tuning(self):
        return sl_batch_tuning(self.h)

    def get(self, sample, slot):
        """(spins of the slot in natural order, temperature index it holds)."""
        out = np.empty(self.L[sample] ** self.d, np.int8)
        k = sl_batch_get(self.h, sample, slot, out)
        return out, k

    def bonds(self, sample):
        out = np.empty((self.d, self.L[sample] ** self.d), np.int8)
        sl_batch_get_bonds(self.h, sample, out)
        return out

    def sweeps_done(self):
        return sl_batch_sweeps_done(self.h)

    def save(self):
        """Checkpoint: per sample (spins [slot][N], slot of each temperature),
        and the sweeps done."""
        state = []
        for s in range(self.nsamples):
            spins, perm = [], np.zeros(self.ntemps, np.int32)
            for r in range(self.ntemps):
                sp, k = self.get(s, r)
                spins.append(sp)
                perm[k] = r
            state.append((np.stack(spins), perm))
        return state, self.sweeps_done()

    def load(self, ckpt):
        state, t = ckpt
        for s, (spins, perm) in enumerate(state):
            sl_batch_set(self.h, s, np.ascontiguousarray(spins, np.int8), perm)
        sl_batch_set_sweeps_done(self.h, t)
