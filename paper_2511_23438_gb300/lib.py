"""Thin ctypes binding of libmpsgb (include/mpsgb.h); argument marshalling only.

Every compute step runs in the CUDA library.  If the library is missing this
module raises instead of falling back to anything else.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmpsgb.so")

# enums of include/mpsgb.h
FP64, SPLIT_TF32X3, SPLIT_BF16X3, FP32 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "split_tf32x3": SPLIT_TF32X3, "split_bf16x3": SPLIT_BF16X3, "fp32": FP32}
ROUTE_MPO, ROUTE_SWAP = 0, 1
LATTICE_2D_GROUPED, LATTICE_3D_SITES, LATTICE_2D_SITES = 0, 1, 2
LAYER_X, LAYER_ZZ, LAYER_ZSTAG = 0, 1, 2
Z_TOT, Z_TOT2, X_TOT, X_STAG2 = 0, 1, 2, 3
MODEL_TFIM, MODEL_XY = 0, 1
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ETIMEDOUT", -4: "EDEVICE", -5: "ESTATE"}


class MpsgbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("chi_max", ctypes.c_int), ("theta", ctypes.c_double),
                ("prec", ctypes.c_int), ("route", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("J", ctypes.c_double), ("h", ctypes.c_double), ("dt", ctypes.c_double),
                ("trotter_order", ctypes.c_int), ("lattice", ctypes.c_int), ("Lz", ctypes.c_int), ("model", ctypes.c_int)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


_lib = None

_SIGS = {
    "mpsgb_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Allocator), ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_void_p)]),
    "mpsgb_apply_layer": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]),
    "mpsgb_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int]),
    "mpsgb_truncate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "mpsgb_expect": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "mpsgb_observables": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "mpsgb_fidelity": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "mpsgb_singular_values": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "mpsgb_bond_dims": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
    "mpsgb_footprint_bytes": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_size_t)]),
    "mpsgb_batch_step": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mpsgb_apply_gates": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double]),
    "mpsgb_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "mpsgb_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(Allocator), ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p)]),
    "mpsgb_destroy": (None, [ctypes.c_void_p]),
    "mpsgb_last_error": (ctypes.c_char_p, []),
    "mpsgb_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    "mpsgb_launch_count": (ctypes.c_ulonglong, []),
    "mpsgb_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]),
    "mpsgb_set_wait_limit": (ctypes.c_longlong, [ctypes.c_longlong]),
    "mpsgb_schedule_info": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]),
    "mpsgb_schedule_gates": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]),
    "mpsgb_kernel_timing": (ctypes.c_int, [ctypes.c_int]),
    "mpsgb_kernel_times": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.POINTER(ctypes.c_double)]),
    "mpsgb_kernel_site_name": (ctypes.c_char_p, [ctypes.c_int]),
    "mpsgb_tc_gemm_selftest": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_double)]),
    "mpsgb_eig_selftest": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                                          ctypes.POINTER(ctypes.c_double)]),
    "mpsgb_svd_selftest": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "mpsgb_eigh_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]),
    "mpsgb_initial_theta": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "mpsgb_gamma_fit_lattice": (ctypes.c_double, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mpsgb_initial_theta_lattice": (ctypes.c_double, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "mpsgb_config_schedule_info": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_longlong)]),
    "mpsgb_config_schedule_gates": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_int)]),
    "mpsgb_gamma_fit": (ctypes.c_double, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mpsgb_rescale": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_double)]),
}


def exported_symbols():
    """Names declared in include/mpsgb.h that this binding wraps."""
    return list(_SIGS)


def load(path=None):
    """Load libmpsgb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libmpsgb.so not found at %s: build it with paper_2511_23438_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise MpsgbError(status, load().mpsgb_last_error().decode())


def config(Lx, Ly, chi, theta, prec="fp64", J=-1.0, h=2.0, dt=0.25, order=2, seed=0, route=ROUTE_MPO,
           lattice=LATTICE_2D_GROUPED, Lz=1, model=MODEL_TFIM):
    return Config(Lx, Ly, chi, theta, PRECISIONS[prec] if isinstance(prec, str) else prec, route, seed, J, h, dt, order,
                  lattice, Lz, model)


def xy_config(Lx, Ly, chi, g, dt, prec="fp64"):
    """The XY workload's config: open Lx x Ly grid, one qubit per site, SWAP routing, second order."""
    return config(Lx, Ly, chi, 0.0, prec=prec, J=g, h=0.0, dt=dt, order=2, route=ROUTE_SWAP,
                  lattice=LATTICE_2D_SITES, model=MODEL_XY)


def convert_checkpoint(src, dst, prec):
    """Rewrite a checkpoint of mpsgb_save for another precision form (FP64 <-> complex64 forms):
    the same state, config and counters, blocks stored in the other element type."""
    import numpy as np
    import struct

    with open(src, "rb") as fh:
        raw = fh.read()
    n_cfg = ctypes.sizeof(Config)
    if raw[:8] != b"MPSGBv2\0":
        raise ValueError("not an mpsgb checkpoint: %s" % src)
    cfg = Config.from_buffer_copy(raw[8:8 + n_cfg])
    off = 8 + n_cfg
    elem, nblk, centre, zero = struct.unpack_from("4i", raw, off)
    off += 16
    head = raw[off:off + 8 + 40]
    off += 48
    dims = struct.unpack_from("%di" % (nblk - 1), raw, off)
    off += 4 * (nblk - 1)
    body = np.frombuffer(raw, dtype=np.complex128 if elem == 8 else np.complex64, offset=off)
    cfg.prec = PRECISIONS[prec] if isinstance(prec, str) else prec
    out_t = np.complex128 if cfg.prec == FP64 else np.complex64
    with open(dst, "wb") as fh:
        fh.write(b"MPSGBv2\0")
        fh.write(bytes(cfg))
        fh.write(struct.pack("4i", 8 if out_t == np.complex128 else 4, nblk, centre, zero))
        fh.write(head)
        fh.write(struct.pack("%di" % (nblk - 1), *dims))
        fh.write(body.astype(out_t).tobytes())


def torch_allocator():
    """An mpsgb_allocator backed by PyTorch's caching allocator (keep the returned object alive)."""
    import torch

    def _alloc(size, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a = Allocator(_ALLOC_FN(_alloc), _FREE_FN(_free), None)
    a._keep = (_alloc, _free)
    return a


def tc_gemm_selftest(M, N, K, mode=0, seed=1, tf32=False):
    mode = mode | (4 if tf32 else 0)
    e = ctypes.c_double()
    _check(load().mpsgb_tc_gemm_selftest(M, N, K, mode, seed, ctypes.byref(e)))
    return e.value


def eig_selftest(n, fp64=True, seed=1, kind=0):
    out = (ctypes.c_double * 6)()
    _check(load().mpsgb_eig_selftest(n, 1 if fp64 else 0, kind, seed, out))
    return dict(zip(("sweeps", "ms", "residual", "orthogonality", "sorted", "wmax"), list(out)))


def svd_selftest(X, fp64=True):
    """One-sided Jacobi SVD of the host complex matrix X on the GPU: (s, metrics)."""
    import numpy as np
    X = np.ascontiguousarray(X, dtype=np.complex128)
    p, q = X.shape
    xs = X.view(np.float64).reshape(-1)
    s = (ctypes.c_double * p)()
    out = (ctypes.c_double * 6)()
    _check(load().mpsgb_svd_selftest(p, q, 1 if fp64 else 0, xs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     s, out))
    return np.array(list(s)), dict(zip(("sweeps", "ms", "residual", "orth_u", "orth_v", "rank"), list(out)))


def eigh_noalloc(n, fp64, A_ptr, lda, w_ptr, V_ptr, ldv, stream=0):
    """Hermitian eigendecomposition of a caller-owned device matrix without any allocation
    (device pointers as ints; see mpsgb_eigh_noalloc in include/mpsgb.h)."""
    _check(load().mpsgb_eigh_noalloc(n, 1 if fp64 else 0, A_ptr, lda, w_ptr, V_ptr, ldv, stream))


def set_wait_limit(cycles):
    """Cycle limit of the library's bounded device waits (<= 0 restores the default); returns the
    previous limit.  See mpsgb_set_wait_limit in include/mpsgb.h."""
    return load().mpsgb_set_wait_limit(int(cycles))


def initial_theta(J, h, dtheta, lattice=None):
    if lattice is None:
        return load().mpsgb_initial_theta(J, h, dtheta)
    return load().mpsgb_initial_theta_lattice(lattice, J, h, dtheta)


def gamma_fit(temperature, chi, n, lattice=None):
    if lattice is None:
        return load().mpsgb_gamma_fit(temperature, chi, n)
    return load().mpsgb_gamma_fit_lattice(lattice, temperature, chi, n)


def rescale(z, z2, F, gamma):
    out = (ctypes.c_double * 2)()
    _check(load().mpsgb_rescale(z, z2, F, gamma, out))
    return out[0], out[1]


def schedule_info(Lx, Ly=None):
    """Schedule facts of an Lx x Ly grid, or of the lattice of a Config passed as the first argument."""
    out = (ctypes.c_longlong * 6)()
    if isinstance(Lx, Config):
        _check(load().mpsgb_config_schedule_info(ctypes.byref(Lx), out))
    else:
        _check(load().mpsgb_schedule_info(Lx, Ly, out))
    keys = ("blocks", "zz_bonds", "intra", "inter", "truncations", "dmax")
    return dict(zip(keys, list(out)))


def schedule_gates(Lx, Ly=None):
    """Inter-block gates in application order, of an Lx x Ly grid or of a Config's lattice."""
    n = ctypes.c_int()
    if isinstance(Lx, Config):
        def query(buf, cap):
            _check(load().mpsgb_config_schedule_gates(ctypes.byref(Lx), buf, cap, ctypes.byref(n)))
    else:
        def query(buf, cap):
            _check(load().mpsgb_schedule_gates(Lx, Ly, buf, cap, ctypes.byref(n)))
    query(None, 0)
    buf = (ctypes.c_int * (6 * n.value))()
    query(buf, n.value)
    v = list(buf)
    return [tuple(v[6 * i: 6 * i + 6]) for i in range(n.value)]


def footprint_bytes(cfg):
    b = ctypes.c_size_t()
    _check(load().mpsgb_footprint_bytes(ctypes.byref(cfg), ctypes.byref(b)))
    return b.value


def launch_count():
    return load().mpsgb_launch_count()


KERNEL_SITES = 11


def kernel_timing(enable):
    _check(load().mpsgb_kernel_timing(1 if enable else 0))


def kernel_times():
    """{site name: (device ms, launches, work)} for every launch site."""
    out = {}
    for s in range(KERNEL_SITES):
        ms, n, w = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
        _check(load().mpsgb_kernel_times(s, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)))
        out[load().mpsgb_kernel_site_name(s).decode()] = (ms.value, n.value, w.value)
    return out


class MPS:
    """One device-resident MPS (an mpsgb handle)."""

    def __init__(self, cfg, stream=None, allocator=None, _handle=None):
        self.cfg = cfg
        self._alloc = allocator
        if _handle is not None:
            self.h = _handle
            return
        h = ctypes.c_void_p()
        _check(load().mpsgb_create(ctypes.byref(cfg), ctypes.byref(allocator) if allocator else None,
                                   ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h

    @classmethod
    def load_checkpoint(cls, path, stream=None, allocator=None):
        h = ctypes.c_void_p()
        _check(load().mpsgb_load(path.encode(), ctypes.byref(allocator) if allocator else None,
                                 ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        return cls(None, _handle=h, allocator=allocator)

    def close(self):
        if getattr(self, "h", None):
            load().mpsgb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_layer(self, layer, angle):
        _check(load().mpsgb_apply_layer(self.h, layer, angle))

    def apply_gates(self, first, count, phi):
        _check(load().mpsgb_apply_gates(self.h, first, count, phi))

    def step(self, J, h, dt, order=2, nsteps=1):
        _check(load().mpsgb_step(self.h, J, h, dt, order, nsteps))

    def truncate(self, chi):
        _check(load().mpsgb_truncate(self.h, chi))

    def observables(self):
        out = (ctypes.c_double * 4)()
        _check(load().mpsgb_observables(self.h, out))
        return {"Z": out[0], "Z2": out[1], "X": out[2], "norm": out[3]}

    def expect(self, obs):
        v = ctypes.c_double()
        _check(load().mpsgb_expect(self.h, obs, ctypes.byref(v)))
        return v.value

    def fidelity(self):
        v = ctypes.c_double()
        _check(load().mpsgb_fidelity(self.h, ctypes.byref(v)))
        return v.value

    def singular_values(self, bond):
        n = ctypes.c_int()
        _check(load().mpsgb_singular_values(self.h, bond, None, 0, ctypes.byref(n)))
        buf = (ctypes.c_double * max(1, n.value))()
        _check(load().mpsgb_singular_values(self.h, bond, buf, n.value, ctypes.byref(n)))
        return list(buf)[: n.value]

    def bond_dims(self):
        n = ctypes.c_int()
        _check(load().mpsgb_bond_dims(self.h, None, 0, ctypes.byref(n)))
        buf = (ctypes.c_int * max(1, n.value))()
        _check(load().mpsgb_bond_dims(self.h, buf, n.value, ctypes.byref(n)))
        return list(buf)[: n.value]

    def stats(self):
        out = (ctypes.c_longlong * 5)()
        _check(load().mpsgb_stats(self.h, out))
        return dict(zip(("truncations", "gates", "centre_moves", "eig_calls", "eig_sweeps"), list(out)))

    def counters(self):
        """All counters (mpsgb_counters): truncations, gates, centre moves, eigensolver / SVD calls and
        sweeps, Cholesky factorisations and Cholesky fallbacks."""
        out = (ctypes.c_longlong * 16)()
        n = ctypes.c_int()
        _check(load().mpsgb_counters(self.h, out, 16, ctypes.byref(n)))
        keys = ("truncations", "gates", "centre_moves", "eig_calls", "eig_sweeps", "chol_ok", "chol_fallbacks")
        return dict(zip(keys, list(out)[: n.value]))

    def save(self, path):
        _check(load().mpsgb_save(self.h, path.encode()))


def batch_step(mps_list, nlayers, use_graph=1):
    """nlayers Trotter steps of every handle, concurrently (mpsgb_batch_step); use_graph = 1 replays
    the fixed launch sequences as CUDA graphs on handles with a stream of their own."""
    arr = (ctypes.c_void_p * len(mps_list))(*[m.h.value if isinstance(m.h, ctypes.c_void_p) else m.h
                                              for m in mps_list])
    _check(load().mpsgb_batch_step(arr, len(mps_list), nlayers, use_graph))
