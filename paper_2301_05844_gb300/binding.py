"""ctypes binding of libbbp.so (the C ABI in include/bbp.h).

Argument marshalling only: every step of blockBP runs in the CUDA library.  The raw
functions keep their C names (``lib().bbp_sweep`` ...); ``Lattice`` wraps a handle.
``lib()`` raises if the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbbp.so")

OK, NOT_CONVERGED = 0, 1
ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NUMERIC, ERR_STATE = -1, -2, -3, -4, -5, -6
OBC, INFINITE = 0, 1
F64, C128, F32, C64 = 0, 1, 2, 3
PREC_FP64, PREC_TF32, PREC_BF16, PREC_TF32X3, PREC_BF16X3 = 0, 1, 2, 3, 4
LEFT, RIGHT, UP, DOWN = 0, 1, 2, 3

_NP_DTYPE = {F64: np.float64, C128: np.complex128, F32: np.float32, C64: np.complex64}
_PREC = {"fp64": PREC_FP64, "tf32": PREC_TF32, "bf16": PREC_BF16, "tf32x3": PREC_TF32X3, "bf16x3": PREC_BF16X3}


class Desc(C.Structure):
    _fields_ = [
        ("Lx", C.c_int), ("Ly", C.c_int), ("boundary", C.c_int), ("d", C.c_int), ("D", C.c_int),
        ("bx", C.c_int), ("by", C.c_int), ("chi", C.c_int), ("chi_exp", C.c_int),
        ("dtype", C.c_int), ("prec", C.c_int), ("tol", C.c_double), ("max_sweeps", C.c_int),
        ("stop_relative", C.c_int), ("fit_tol", C.c_double), ("fit_max_sweeps", C.c_int),
        ("seed", C.c_ulonglong), ("init_mode", C.c_int), ("warm_start", C.c_int),
        ("hermitian_basis", C.c_int), ("stream", C.c_void_p), ("single_layer", C.c_int),
        ("shift_x", C.c_int), ("shift_y", C.c_int), ("launch_mode", C.c_int), ("keep_fp64", C.c_int),
    ]


class StepTime(C.Structure):
    _fields_ = [
        ("index", C.c_int), ("kernel_class", C.c_int), ("tasks", C.c_int), ("tile_n", C.c_int),
        ("max_m", C.c_longlong), ("max_n", C.c_longlong), ("max_k", C.c_longlong),
        ("flops", C.c_double), ("bytes", C.c_double), ("ms", C.c_double),
    ]


class Term(C.Structure):
    _fields_ = [
        ("nsite", C.c_int), ("site", C.c_int * 2),
        ("op_re", C.POINTER(C.c_double) * 2), ("op_im", C.POINTER(C.c_double) * 2),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("flops", C.c_double), ("qr_flops", C.c_double), ("kernels", C.c_longlong),
        ("fit_sweeps", C.c_longlong), ("fits", C.c_longlong), ("sweeps", C.c_int),
        ("last_residual", C.c_double), ("first_residual", C.c_double), ("fit_loop_iters", C.c_longlong),
    ]


_lib = None


def lib():
    """Load libbbp.so (raises FileNotFoundError if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FileNotFoundError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    L.bbp_create_lattice.argtypes = [C.POINTER(Desc), C.POINTER(P)]
    L.bbp_set_tensors.argtypes = [P, P, C.c_int]
    L.bbp_sweep.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.bbp_expect.argtypes = [P, C.POINTER(Term), C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.bbp_destroy.argtypes = [P]
    L.bbp_rdm.argtypes = [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.bbp_destroy.restype = None
    L.bbp_last_error.restype = C.c_char_p
    L.bbp_get_message.argtypes = [P, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.bbp_set_message.argtypes = [P, C.c_int, C.c_int, C.POINTER(C.c_double)]
    L.bbp_get_stats.argtypes = [P, C.POINTER(Stats)]
    L.bbp_time_kernels.argtypes = [P, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.bbp_selftest_gemm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, P, P, P]
    L.bbp_selftest_rng.argtypes = [C.c_ulonglong, C.c_ulonglong, C.c_longlong, P]
    L.bbp_qr_batched.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, P]
    L.bbp_qr_batched_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, P]
    L.bbp_lattice_footprint.argtypes = [C.POINTER(Desc), C.POINTER(C.c_size_t)]
    L.bbp_autotune.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.bbp_time_steps.argtypes = [P, C.c_int, C.c_int, C.POINTER(StepTime), C.POINTER(C.c_int)]
    L.bbp_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(P)]
    L.bbp_server_submit.argtypes = [P, C.POINTER(Desc), P, C.POINTER(Term), C.c_int, C.POINTER(C.c_longlong)]
    L.bbp_server_poll.argtypes = [P, C.c_longlong, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]
    L.bbp_server_wait.argtypes = [P, C.c_longlong, C.c_double]
    L.bbp_server_stats.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_size_t)]
    L.bbp_server_destroy.argtypes = [P]
    L.bbp_server_destroy.restype = None
    _lib = L
    return L


class BBPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bbp error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc < 0:
        raise BBPError(rc, lib().bbp_last_error().decode())
    return rc


def make_desc(Lx, Ly, d, D, bx, by, chi, boundary="obc", chi_exp=0, dtype=F64, prec="fp64", tol=1e-5,
              max_sweeps=10, stop_relative=0, fit_tol=1e-6, fit_max_sweeps=10, seed=0, init_mode=0, warm_start=0,
              hermitian_basis=0, stream=None, single_layer=0, shift=(0, 0), launch_mode=0, keep_fp64=0):
    return Desc(Lx, Ly, OBC if boundary == "obc" else INFINITE, d, D, bx, by, chi, chi_exp, dtype,
                _PREC[prec] if isinstance(prec, str) else prec, tol, max_sweeps, stop_relative, fit_tol,
                fit_max_sweeps, seed, init_mode, int(warm_start), int(hermitian_basis), stream, int(single_layer),
                int(shift[0]), int(shift[1]), int(launch_mode), int(keep_fp64))


def _term_array(terms):
    """ctypes bbp_term array for [(site, op), ...] terms, plus the arrays it points into."""
    n = len(terms)
    arr = (Term * max(n, 1))()
    keep = []
    for i, term in enumerate(terms):
        arr[i].nsite = len(term)
        for k, (s, op) in enumerate(term):
            op = np.asarray(op)
            re = np.ascontiguousarray(op.real, dtype=np.float64)
            im = np.ascontiguousarray(op.imag, dtype=np.float64) if np.iscomplexobj(op) else None
            keep += [re, im]
            arr[i].site[k] = s
            arr[i].op_re[k] = re.ctypes.data_as(C.POINTER(C.c_double))
            arr[i].op_im[k] = im.ctypes.data_as(C.POINTER(C.c_double)) if im is not None else None
    return arr, keep


def _flat_tensors(tensors, dtype):
    dt = _NP_DTYPE[dtype]
    return np.concatenate([np.ascontiguousarray(t, dtype=dt).reshape(-1) for t in tensors])


def footprint(**kw):
    """Resident device bytes of a lattice with this description (no allocation)."""
    desc = make_desc(**kw)
    b = C.c_size_t()
    _check(lib().bbp_lattice_footprint(C.byref(desc), C.byref(b)))
    return b.value


class Server:
    """Owning wrapper of a bbp_server (continuous batching of whole solves)."""

    QUEUED, RUNNING, DONE = 0, 1, 2

    def __init__(self, max_bytes, max_active=64):
        self.h = C.c_void_p()
        _check(lib().bbp_server_create(int(max_bytes), int(max_active), C.byref(self.h)))
        self._nterms = {}

    def submit(self, tensors, terms=(), **kw):
        desc = make_desc(**kw)
        flat = _flat_tensors(tensors, desc.dtype)
        arr, _keep = _term_array(list(terms))
        rid = C.c_longlong()
        _check(lib().bbp_server_submit(self.h, C.byref(desc), flat.ctypes.data_as(C.c_void_p), arr, len(terms),
                                       C.byref(rid)))
        self._nterms[rid.value] = len(terms)
        return rid.value

    def poll(self, rid):
        """dict(state, values (complex array once done), sweeps, residual, latency_s)."""
        n = self._nterms[rid]
        st, k = C.c_int(), C.c_int()
        res, lat = C.c_double(), C.c_double()
        re, im = np.zeros(max(n, 1)), np.zeros(max(n, 1))
        _check(lib().bbp_server_poll(self.h, rid, C.byref(st), re.ctypes.data_as(C.POINTER(C.c_double)),
                                     im.ctypes.data_as(C.POINTER(C.c_double)), C.byref(k), C.byref(res),
                                     C.byref(lat)))
        return dict(state=st.value, values=(re + 1j * im)[:n] if st.value == self.DONE else None,
                    sweeps=k.value, residual=res.value, latency_s=lat.value)

    def wait(self, rid, timeout_s=600.0):
        _check(lib().bbp_server_wait(self.h, rid, float(timeout_s)))
        return self.poll(rid)

    def stats(self):
        a, b, c = C.c_longlong(), C.c_longlong(), C.c_longlong()
        u = C.c_size_t()
        _check(lib().bbp_server_stats(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(u)))
        return dict(submitted=a.value, done=b.value, sweeps=c.value, bytes_in_use=u.value)

    def close(self):
        if self.h:
            lib().bbp_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def expect_centred(lattices, terms):
    """<O> of every term from the partition (one of `lattices`, the same OBC lattice run with
    different shifts) in which its sites lie deepest inside one block; returns (values,
    index of the lattice each term was read from)."""
    n = len(terms)
    arr, keep = _term_array(terms)
    hs = (C.c_void_p * len(lattices))(*[g.h.value for g in lattices])
    out_re, out_im, chosen = np.zeros(n), np.zeros(n), np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().bbp_expect_centred(hs, len(lattices), arr, n, out_re.ctypes.data_as(C.POINTER(C.c_double)),
                                    out_im.ctypes.data_as(C.POINTER(C.c_double)),
                                    chosen.ctypes.data_as(C.POINTER(C.c_int))))
    return out_re + 1j * out_im, chosen[:n]


class Lattice:
    """Owning wrapper of a bbp_lattice handle."""

    def __init__(self, **kw):
        self.desc = make_desc(**kw)
        self.h = C.c_void_p()
        _check(lib().bbp_create_lattice(C.byref(self.desc), C.byref(self.h)))

    def close(self):
        if self.h:
            lib().bbp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tensors(self, tensors=None, device_ptr=None, host_ptr=None):
        """tensors: list of numpy arrays T[p,u,l,d,r] (E[u,l,d,r] on a single-layer network;
        cast to the desc dtype); or device_ptr / host_ptr: the address of the same data,
        already in the desc dtype and concatenated, on the GPU / in (pinned) host memory."""
        if device_ptr is not None:
            return _check(lib().bbp_set_tensors(self.h, C.c_void_p(device_ptr), 1))
        if host_ptr is not None:
            return _check(lib().bbp_set_tensors(self.h, C.c_void_p(host_ptr), 0))
        flat = _flat_tensors(tensors, self.desc.dtype)
        self._host = flat
        return _check(lib().bbp_set_tensors(self.h, flat.ctypes.data_as(C.c_void_p), 0))

    def sweep(self, n=0):
        r = C.c_double()
        k = C.c_int()
        rc = _check(lib().bbp_sweep(self.h, n, C.byref(r), C.byref(k)))
        return r.value, k.value, rc

    def expect(self, terms):
        """terms: list of [(site, op), ...] with d x d numpy operators (on a single-layer
        network, the impurity tensors that replace the site tensors)."""
        n = len(terms)
        arr, keep = _term_array(terms)
        out_re = np.zeros(n)
        out_im = np.zeros(n)
        _check(lib().bbp_expect(self.h, arr, n, out_re.ctypes.data_as(C.POINTER(C.c_double)),
                                out_im.ctypes.data_as(C.POINTER(C.c_double))))
        return out_re + 1j * out_im

    def rdm(self, sites):
        """Reduced density matrix (d^n x d^n complex, n = len(sites) = 1 or 2) of the sites."""
        n = len(sites)
        dim = self.desc.d ** n
        s = (C.c_int * 2)(*sites, *([0] * (2 - n)))
        re, im = np.zeros(dim * dim), np.zeros(dim * dim)
        _check(lib().bbp_rdm(self.h, n, s, re.ctypes.data_as(C.POINTER(C.c_double)),
                             im.ctypes.data_as(C.POINTER(C.c_double))))
        return (re + 1j * im).reshape(dim, dim)

    def get_message(self, block, direction):
        ns = C.c_int()
        bonds = (C.c_int * 64)()
        _check(lib().bbp_get_message(self.h, block, direction, C.byref(ns), bonds, None))
        b = [bonds[i] for i in range(ns.value + 1)]
        K = self.desc.D if self.desc.single_layer else self.desc.D ** 2
        cplx = self.complex_messages()
        total = sum(b[i] * K * b[i + 1] for i in range(ns.value)) * (2 if cplx else 1)
        buf = np.zeros(total)
        _check(lib().bbp_get_message(self.h, block, direction, None, None, buf.ctypes.data_as(C.POINTER(C.c_double))))
        if cplx:
            buf = buf[0::2] + 1j * buf[1::2]
        out, o = [], 0
        for i in range(ns.value):
            n = b[i] * K * b[i + 1]
            out.append(buf[o:o + n].reshape(b[i], K, b[i + 1]))
            o += n
        return out

    def complex_messages(self):
        """False when the lattice runs in real arithmetic (real tensors, or complex ones in
        the Hermitian basis)."""
        d = self.desc
        return d.dtype in (C128, C64) and d.prec == PREC_FP64 and not d.hermitian_basis

    def time_steps(self, reps=3):
        """Every launch of the planned sweep timed on its own (bbp_time_steps): a list of dicts."""
        n = C.c_int()
        _check(lib().bbp_time_steps(self.h, reps, 0, None, C.byref(n)))
        rows = (StepTime * max(n.value, 1))()
        _check(lib().bbp_time_steps(self.h, reps, n.value, rows, C.byref(n)))
        return [{f: getattr(r, f) for f, _ in StepTime._fields_} for r in rows[:n.value]]

    def autotune(self, reps=3):
        """Choose the tensor-core tile shapes of the planned sweep by timing them (before
        the first sweep).  Returns (ms_before, ms_after, steps_changed)."""
        a, b, k = C.c_double(), C.c_double(), C.c_int()
        _check(lib().bbp_autotune(self.h, int(reps), C.byref(a), C.byref(b), C.byref(k)))
        return a.value, b.value, k.value

    def stats(self):
        s = Stats()
        _check(lib().bbp_get_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}
