"""Thin ctypes binding of libtcm.so (include/tcm.h), with the same names as the C ABI.

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  PyTorch supplies device memory and the stream.  Loading fails
loudly (``TcmError``) when the library has not been built; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtcm.so")

TCM_OK, TCM_EINVAL, TCM_ENOTCONV, TCM_ENOMEM, TCM_ECUDA, TCM_ETIMEOUT = range(6)
TCM_F32, TCM_F64 = 0, 1
TCM_FP64, TCM_MIXED = 0, 1
LMAX_MAX = 24
PHASES = ("geom", "moments", "finalize", "contract", "direct", "host")
NPHASES = len(PHASES)
_NAMES = {0: "TCM_OK", 1: "TCM_EINVAL", 2: "TCM_ENOTCONV", 3: "TCM_ENOMEM", 4: "TCM_ECUDA", 5: "TCM_ETIMEOUT"}


class TcmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class tcm_system(ctypes.Structure):
    _fields_ = [("xyzq", ctypes.c_void_p), ("n", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("has_center", ctypes.c_int32), ("center", ctypes.c_double * 3), ("radius", ctypes.c_double),
                ("moments", ctypes.c_void_p), ("moments_lmax", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class tcm_moments_t(ctypes.Structure):
    _fields_ = [("q", ctypes.c_void_p), ("lmax", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("center", ctypes.c_double * 3), ("radius", ctypes.c_double)]


class tcm_pair_item(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int32), ("b", ctypes.c_int32), ("lmax", ctypes.c_int32), ("has_rot", ctypes.c_int32),
                ("rotB", ctypes.c_double * 9), ("R0", ctypes.c_double * 3)]


PAIR_ITEM_DTYPE = np.dtype([("a", "<i4"), ("b", "<i4"), ("lmax", "<i4"), ("has_rot", "<i4"),
                            ("rotB", "<f8", (9,)), ("R0", "<f8", (3,))])
assert PAIR_ITEM_DTYPE.itemsize == ctypes.sizeof(tcm_pair_item)

_lib = None


def lib():
    """Load libtcm.so (once).  Raises TcmError if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise TcmError(TCM_ECUDA, f"{LIB_PATH} is not built; run paper_0704_1672_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.tcm_ctx_create.argtypes = [ctypes.POINTER(P), i32, P]
        L.tcm_ctx_destroy.argtypes = [P]
        L.tcm_ctx_destroy.restype = None
        L.tcm_ctx_set_stream.argtypes = [P, P]
        L.tcm_last_error.restype = ctypes.c_char_p
        L.tcm_prepare.argtypes = [P, ctypes.POINTER(tcm_system)]
        L.tcm_moments.argtypes = [P, ctypes.POINTER(tcm_system), P, i32, i32, ctypes.POINTER(tcm_moments_t)]
        L.tcm_energy.argtypes = [P, ctypes.POINTER(tcm_moments_t), ctypes.POINTER(tcm_moments_t), P, i32,
                                 ctypes.POINTER(d)]
        L.tcm_energy_batch.argtypes = [P, i32, P, i64, P, i32, P, P]
        L.tcm_direct.argtypes = [P, ctypes.POINTER(tcm_system), ctypes.POINTER(tcm_system), P, P, ctypes.POINTER(d)]
        L.tcm_moments_noalloc.argtypes = [ctypes.POINTER(tcm_system), P, i32, i32, P, P, P]
        L.tcm_ctx_set_profiling.argtypes = [P, i32]
        L.tcm_ctx_set_tiling.argtypes = [P, i32, i32]
        L.tcm_ctx_set_tiling_l.argtypes = [P, i32, i32, i32, i32]
        L.tcm_ctx_get_tiling_l.argtypes = [P, i32, i32, P, P]
        L.tcm_ctx_set_chunking_l.argtypes = [P, i32, i32]
        L.tcm_ctx_get_chunking_l.argtypes = [P, i32, P, P]
        L.tcm_ctx_set_graphs.argtypes = [P, i32]
        L.tcm_ctx_set_rotate_cached.argtypes = [P, i32]
        L.tcm_gradients_batch.argtypes = [P, i32, P, ctypes.c_int64, P, i32, P, P, P]
        L.tcm_direct_batch.argtypes = [P, P, P, ctypes.c_int64, P, P, P]
        L.tcm_rotate_moments.argtypes = [P, ctypes.c_int64, P, P, P]
        L.tcm_ctx_graph_stats.argtypes = [P, P, P]
        L.tcm_ctx_read_profile.argtypes = [P, P, P]
        for name in ("tcm_ctx_create", "tcm_ctx_set_stream", "tcm_prepare", "tcm_moments", "tcm_energy",
                     "tcm_energy_batch", "tcm_direct", "tcm_ctx_set_profiling", "tcm_ctx_read_profile",
                     "tcm_moments_noalloc", "tcm_ctx_set_tiling", "tcm_ctx_set_graphs", "tcm_ctx_graph_stats",
                     "tcm_ctx_set_tiling_l", "tcm_ctx_get_tiling_l", "tcm_ctx_set_chunking_l", "tcm_ctx_get_chunking_l",
                     "tcm_ctx_set_rotate_cached", "tcm_rotate_moments", "tcm_gradients_batch",
                     "tcm_direct_batch"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(rc):
    if rc != TCM_OK:
        raise TcmError(rc, lib().tcm_last_error().decode())


def _dptr(arr):
    """Host pointer of a contiguous float64 numpy array (or None)."""
    if arr is None:
        return None
    return arr.ctypes.data_as(ctypes.c_void_p)


def make_system(xyzq: torch.Tensor, center=None, radius=None, moments: "MomentSet | None" = None) -> tcm_system:
    """Descriptor of one device-resident system: (N, 4) float32 or float64 records (x, y, z, q).

    ``moments`` (from tcm_moments about the same centre) is a device cache that batches use for the
    system's unrotated sides."""
    if not isinstance(xyzq, torch.Tensor) or not xyzq.is_cuda:
        raise TcmError(TCM_EINVAL, "coordinates must be a CUDA tensor")
    if xyzq.dim() != 2 or xyzq.shape[1] != 4 or not xyzq.is_contiguous():
        raise TcmError(TCM_EINVAL, "coordinates must be a contiguous (N, 4) tensor")
    if xyzq.dtype == torch.float32:
        dt = TCM_F32
    elif xyzq.dtype == torch.float64:
        dt = TCM_F64
    else:
        raise TcmError(TCM_EINVAL, "coordinates must be float32 or float64")
    s = tcm_system()
    s.xyzq = xyzq.data_ptr() if xyzq.numel() else None
    s.n = xyzq.shape[0]
    s.dtype = dt
    if center is not None:
        s.has_center = 1
        for k in range(3):
            s.center[k] = float(center[k])
    s.radius = -1.0 if radius is None else float(radius)
    if moments is not None:
        s.moments = moments.q.data_ptr()
        s.moments_lmax = moments.lmax
    return s


@dataclass
class MomentSet:
    """Packed moments on the device plus the centre and radius they refer to."""
    q: torch.Tensor
    lmax: int
    center: np.ndarray
    radius: float

    def struct(self):
        m = tcm_moments_t()
        m.q = self.q.data_ptr()
        m.lmax = self.lmax
        for k in range(3):
            m.center[k] = float(self.center[k])
        m.radius = float(self.radius)
        return m


class Context:
    """A library context bound to the current CUDA device and a torch stream."""

    def __init__(self, lmax_cap: int = LMAX_MAX, stream: torch.cuda.Stream | None = None):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib().tcm_ctx_create(ctypes.byref(h), int(lmax_cap), ctypes.c_void_p(self.stream.cuda_stream)))
        self._h = h
        self.lmax_cap = lmax_cap

    def close(self):
        if getattr(self, "_h", None):
            lib().tcm_ctx_destroy(self._h)
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

    def tcm_ctx_set_tiling(self, precision, atoms_per_lane):
        _check(lib().tcm_ctx_set_tiling(self._h, int(precision), int(atoms_per_lane)))

    def tcm_ctx_set_tiling_l(self, precision, lmax, atoms_per_lane, ctas_per_sm):
        _check(lib().tcm_ctx_set_tiling_l(self._h, int(precision), int(lmax), int(atoms_per_lane), int(ctas_per_sm)))

    def tcm_ctx_get_tiling_l(self, precision, lmax):
        apl, cps = ctypes.c_int(), ctypes.c_int()
        _check(lib().tcm_ctx_get_tiling_l(self._h, int(precision), int(lmax), ctypes.byref(apl), ctypes.byref(cps)))
        return apl.value, cps.value

    def tcm_ctx_set_chunking_l(self, lmax, kmax):
        _check(lib().tcm_ctx_set_chunking_l(self._h, int(lmax), int(kmax)))

    def tcm_ctx_get_chunking_l(self, lmax):
        """(kmax, number of column chunks) of the mixed path's moment pass at degree lmax."""
        km, nch = ctypes.c_int(), ctypes.c_int()
        _check(lib().tcm_ctx_get_chunking_l(self._h, int(lmax), ctypes.byref(km), ctypes.byref(nch)))
        return km.value, nch.value

    def tcm_ctx_set_rotate_cached(self, enable: bool):
        _check(lib().tcm_ctx_set_rotate_cached(self._h, 1 if enable else 0))

    def tcm_rotate_moments(self, moms, rot, lmax=None, out=None):
        """Moments of rotated systems from their moments (Wigner rotation, no atoms).

        moms: a MomentSet or a list of them; rot: (3, 3) or (n, 3, 3).  Returns MomentSet(s) at
        ``lmax`` (default: each input's lmax); asynchronous on the context stream."""
        single = isinstance(moms, MomentSet)
        ms = [moms] if single else list(moms)
        R = np.ascontiguousarray(np.asarray(rot, dtype=np.float64).reshape(-1, 9))
        if len(R) != len(ms):
            raise TcmError(TCM_EINVAL, "one rotation per moment set")
        outs = [] if out is None else ([out] if single else list(out))
        ins = (tcm_moments_t * max(len(ms), 1))()
        res = (tcm_moments_t * max(len(ms), 1))()
        for i, m in enumerate(ms):
            L = m.lmax if lmax is None else int(lmax)
            if out is None:
                outs.append(MomentSet(torch.empty((L + 1) ** 2, dtype=torch.float64, device=m.q.device), L,
                                      np.array(m.center, dtype=np.float64), float(m.radius)))
            ins[i] = m.struct()
            res[i] = outs[i].struct()
            res[i].lmax = L
        _check(lib().tcm_rotate_moments(self._h, len(ms), ctypes.cast(ins, ctypes.c_void_p),
                                        R.ctypes.data_as(ctypes.c_void_p), ctypes.cast(res, ctypes.c_void_p)))
        for i, o in enumerate(outs):
            o.lmax = res[i].lmax
            o.center = np.array([res[i].center[k] for k in range(3)])
            o.radius = res[i].radius
        return outs[0] if single else outs

    def tcm_ctx_set_graphs(self, mode):
        """0 (or False): launch kernel by kernel; 1 (or True, default): capture a shape seen twice in
        a row; 2: capture every new shape on its first call."""
        _check(lib().tcm_ctx_set_graphs(self._h, int(mode)))

    def tcm_ctx_graph_stats(self):
        cap, lau = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().tcm_ctx_graph_stats(self._h, ctypes.byref(cap), ctypes.byref(lau)))
        return cap.value, lau.value

    def tcm_ctx_set_profiling(self, enable: bool):
        _check(lib().tcm_ctx_set_profiling(self._h, 1 if enable else 0))

    def tcm_ctx_read_profile(self):
        """(ms per phase, kernel launches per phase) since the last read; synchronises the stream."""
        ms = np.zeros(NPHASES)
        launches = np.zeros(NPHASES, dtype=np.int64)
        _check(lib().tcm_ctx_read_profile(self._h, ms.ctypes.data_as(ctypes.c_void_p),
                                          launches.ctypes.data_as(ctypes.c_void_p)))
        return dict(zip(PHASES, ms)), dict(zip(PHASES, launches.tolist()))

    def set_stream(self, stream: torch.cuda.Stream):
        _check(lib().tcm_ctx_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))
        self.stream = stream

    # ---------------------------------------------------------------- a1
    def tcm_prepare(self, xyzq, center=None):
        """Centroid (unless given) and radius of a device system; returns (center, radius)."""
        s = make_system(xyzq, center=center)
        _check(lib().tcm_prepare(self._h, ctypes.byref(s)))
        return np.array(s.center[:]), float(s.radius)

    # ---------------------------------------------------------------- Eq. (multipole)
    def tcm_moments(self, xyzq, lmax, precision=TCM_MIXED, rot=None, center=None, radius=None, out=None) -> MomentSet:
        s = make_system(xyzq, center=center, radius=radius)
        n = (lmax + 1) ** 2
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=xyzq.device)
        m = tcm_moments_t()
        m.q = out.data_ptr()
        r = None if rot is None else np.ascontiguousarray(rot, dtype=np.float64).reshape(9)
        _check(lib().tcm_moments(self._h, ctypes.byref(s), _dptr(r), int(lmax), int(precision), ctypes.byref(m)))
        return MomentSet(out, lmax, np.array(m.center[:]), float(m.radius))

    # ---------------------------------------------------------------- Eq. (Formula)
    def tcm_energy(self, A: MomentSet, B: MomentSet, R0, lmax=None) -> float:
        lmax = min(A.lmax, B.lmax) if lmax is None else lmax
        a, b = A.struct(), B.struct()
        R = np.ascontiguousarray(R0, dtype=np.float64).reshape(3)
        E = ctypes.c_double()
        _check(lib().tcm_energy(self._h, ctypes.byref(a), ctypes.byref(b), _dptr(R), int(lmax), ctypes.byref(E)))
        return E.value

    def tcm_energy_batch(self, systems, a, b, lmax, R0, rotB=None, precision=TCM_MIXED, E=None, status=None):
        """Batched moments + energies.

        systems: list of tcm_system descriptors (``make_system``) or (tensor, center, radius) tuples.
        a, b, lmax: per-item int arrays; R0: (k, 3); rotB: (k, 3, 3) or None.
        Returns (E, status) device tensors; the call is asynchronous on the context stream.
        """
        return self.tcm_energy_batch_packed(pack_batch(systems, a, b, lmax, R0, rotB), precision, E, status)

    def tcm_energy_batch_packed(self, pb: "PackedBatch", precision=TCM_MIXED, E=None, status=None):
        """tcm_energy_batch on arguments already marshalled by ``pack_batch``."""
        k = len(pb.items)
        dev = torch.device("cuda", torch.cuda.current_device())
        if E is None:
            E = torch.empty(k, dtype=torch.float64, device=dev)
        if status is None:
            status = torch.empty(k, dtype=torch.int32, device=dev)
        _check(lib().tcm_energy_batch(self._h, pb.n_systems, ctypes.cast(pb.sys_arr, ctypes.c_void_p), k,
                                      pb.items.ctypes.data_as(ctypes.c_void_p), int(precision),
                                      ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(status.data_ptr())))
        return E, status

    def tcm_gradients_batch(self, systems, a, b, lmax, R0, rotB=None, precision=TCM_MIXED, E=None, G=None,
                            status=None):
        """Batched energies with the force on B and the torques on A and B (lab frame).

        Returns (E, G, status): G is a (k, 9) device tensor [F_B, tau_A, tau_B] per item."""
        pb = pack_batch(systems, a, b, lmax, R0, rotB)
        k = len(pb.items)
        dev = torch.device("cuda", torch.cuda.current_device())
        if E is None:
            E = torch.empty(k, dtype=torch.float64, device=dev)
        if G is None:
            G = torch.empty((k, 9), dtype=torch.float64, device=dev)
        if status is None:
            status = torch.empty(k, dtype=torch.int32, device=dev)
        _check(lib().tcm_gradients_batch(self._h, pb.n_systems, ctypes.cast(pb.sys_arr, ctypes.c_void_p), k,
                                         pb.items.ctypes.data_as(ctypes.c_void_p), int(precision),
                                         ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(G.data_ptr()),
                                         ctypes.c_void_p(status.data_ptr())))
        return E, G, status

    # ---------------------------------------------------------------- Eq. (Coulomb)
    def tcm_direct(self, A, B, R0, rotB=None, cA=None, cB=None) -> float:
        sa = make_system(A, center=cA)
        sb = make_system(B, center=cB)
        R = np.ascontiguousarray(R0, dtype=np.float64).reshape(3)
        r = None if rotB is None else np.ascontiguousarray(rotB, dtype=np.float64).reshape(9)
        E = ctypes.c_double()
        _check(lib().tcm_direct(self._h, ctypes.byref(sa), ctypes.byref(sb), _dptr(r), _dptr(R), ctypes.byref(E)))
        return E.value

    def tcm_direct_batch(self, A, B, R0, rotB=None, cA=None, cB=None, E=None):
        """Eq. (Coulomb) for k placements of B (R0: (k, 3); rotB: (k, 3, 3) or None); returns the
        (k,) device tensor of energies (asynchronous)."""
        sa = make_system(A, center=cA)
        sb = make_system(B, center=cB)
        R = np.ascontiguousarray(R0, dtype=np.float64).reshape(-1, 3)
        k = len(R)
        r = None if rotB is None else np.ascontiguousarray(rotB, dtype=np.float64).reshape(k, 9)
        if E is None:
            E = torch.empty(k, dtype=torch.float64, device=A.device)
        _check(lib().tcm_direct_batch(self._h, ctypes.byref(sa), ctypes.byref(sb), k, _dptr(r), _dptr(R),
                                      ctypes.c_void_p(E.data_ptr())))
        return E


NOALLOC_MAX_ATOMS = 262144


def tcm_moments_noalloc(xyzq, lmax, precision=TCM_MIXED, rot=None, center=None, radius=None, out=None,
                        center_radius_out=None, stream=None):
    """The C entry point that allocates no device memory (for callers that cannot allocate).

    ``out`` (contiguous float64 CUDA tensor of at least (lmax+1)^2 entries) and
    ``center_radius_out`` (contiguous float64 CUDA tensor of at least 4 entries) must be on the
    device of ``xyzq``; such callers pass them preallocated.  The library call itself allocates
    nothing and queues its work on ``stream`` (default: the current torch stream of that
    device).  Calls that overlap on the GPU race on the library's shared scratch, so serialise
    them.
    """
    s = make_system(xyzq, center=center, radius=radius)
    dev = xyzq.device
    if out is None:
        out = torch.empty((lmax + 1) ** 2, dtype=torch.float64, device=dev)

    def _check_out(t, n, what):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or t.device != dev \
                or not t.is_contiguous() or t.numel() < n:
            raise TcmError(TCM_EINVAL, f"{what} must be a contiguous float64 CUDA tensor of at least {n} entries on {dev}")

    _check_out(out, (max(int(lmax), 0) + 1) ** 2, "out")
    if center_radius_out is not None:
        _check_out(center_radius_out, 4, "center_radius_out")
    with torch.cuda.device(dev):
        stream = stream if stream is not None else torch.cuda.current_stream(dev)
        r = None if rot is None else np.ascontiguousarray(rot, dtype=np.float64).reshape(9)
        g = None if center_radius_out is None else ctypes.c_void_p(center_radius_out.data_ptr())
        _check(lib().tcm_moments_noalloc(ctypes.byref(s), _dptr(r), int(lmax), int(precision),
                                         ctypes.c_void_p(out.data_ptr()), g, ctypes.c_void_p(stream.cuda_stream)))
    return out


@dataclass
class PackedBatch:
    """Marshalled arguments of tcm_energy_batch (reusable across calls)."""
    sys_arr: object
    n_systems: int
    items: np.ndarray
    keep: list


def pack_batch(systems, a, b, lmax, R0, rotB=None) -> PackedBatch:
    sys_arr = (tcm_system * max(len(systems), 1))()
    keep = []
    for i, s in enumerate(systems):
        if not isinstance(s, tcm_system):
            t, c, r = s
            s = make_system(t, center=c, radius=r)
            keep.append(t)
        sys_arr[i] = s
    k = len(R0)
    items = np.zeros(k, dtype=PAIR_ITEM_DTYPE)
    items["a"] = a
    items["b"] = b
    items["lmax"] = lmax
    items["R0"] = np.asarray(R0, dtype=np.float64).reshape(k, 3)
    if rotB is not None:
        items["has_rot"] = 1
        items["rotB"] = np.asarray(rotB, dtype=np.float64).reshape(k, 9)
    return PackedBatch(sys_arr, len(systems), items, keep)


def unpack(q, lmax=None):
    """Packed real moments -> complex Q_lm indexed l*l + l + m (m = -l..l), using Q_l,-m = (-1)^m conj(Q_lm)."""
    q = q.detach().cpu().numpy() if isinstance(q, torch.Tensor) else np.asarray(q)
    L = int(round(np.sqrt(len(q)))) - 1 if lmax is None else lmax
    out = np.zeros((L + 1) ** 2, dtype=np.complex128)
    for l in range(L + 1):
        out[l * l + l] = q[l * l]
        for m in range(1, l + 1):
            z = q[l * l + 2 * m - 1] + 1j * q[l * l + 2 * m]
            out[l * l + l + m] = z
            out[l * l + l - m] = (-1) ** m * np.conj(z)
    return out
