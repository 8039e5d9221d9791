"""ctypes binding of liblbx.so (include/lbx.h).  Argument marshalling only: every step
of the kinetic relaxation scheme runs in the library's CUDA kernels.  Importing this
module fails if the library has not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbx.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python {_HERE}/build.py`")
_lib = C.CDLL(LIB_PATH)

# ------------------------------------------------------------------------- constants
ADR_CASCADE, NSF_PRIM_TRACK, MHD_J_TRACK, BURGERS, EULER, MAXWELL_TM = 1, 2, 3, 4, 5, 6
NSF_CONS_TRACK, MHD_POWELL_2D, HCNSF_3D = 7, 8, 9
D2Q5, D2Q9, D3Q7, D3Q19 = 1, 2, 3, 4
ACOUSTIC, DIFFUSIVE = 1, 2
FP64, FP32_SHIFT, FP16_SCALED = 1, 2, 3
MMS_NONE, MMS_ADR_SEPARABLE, MMS_FOURIER = 0, 1, 2
MMS_MAX_MODES = 64
STAGE_AUTO, STAGE_THREAD, STAGE_LANES2, STAGE_BULK, STAGE_PIPE = 0, 1, 2, 3, 4
PRESCRIBED_NONE, PRESCRIBED_UNIFORM, PRESCRIBED_ADVECTED = 0, 1, 2
STREAM_TWO_BUFFERS, STREAM_IN_PLACE = 0, 1

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_SUBCHAR", 5: "ERR_NONFINITE",
          6: "ERR_TIMEOUT", 7: "ERR_STATE", 8: "ERR_IO", 9: "ERR_UNSUPPORTED"}


class LbxError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class SystemDesc(C.Structure):
    _fields_ = [("family", C.c_int), ("params", C.c_double * 8), ("Q0", C.c_double * 24)]


class MmsMode(C.Structure):
    _fields_ = [("p", C.c_int), ("k", C.c_int * 3), ("amp", C.c_double), ("phase", C.c_double),
                ("sigma", C.c_double), ("omega", C.c_double), ("psi", C.c_double)]


class SchemeDesc(C.Structure):
    _fields_ = [("lattice", C.c_int), ("extent", C.c_int64 * 3), ("scaling", C.c_int),
                ("f", C.c_double), ("tau_lb", C.c_double), ("tau_R", C.c_double),
                ("g_tau", C.c_double), ("precision", C.c_int), ("mms", C.c_int),
                ("mms_amp", C.c_double), ("allow_subchar_violation", C.c_int),
                ("mms_modes", C.POINTER(MmsMode)), ("mms_n_modes", C.c_int), ("mms_mean", C.c_double * 8),
                ("mms_conserved_only", C.c_int), ("prescribed", C.c_int),
                ("prescribed_params", C.c_double * 10), ("streaming", C.c_int),
                ("slab_origin", C.c_int64), ("slab_planes_global", C.c_int64),
                ("fp16_scales", C.c_double * 24)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def _sig(name, res, args):
    fn = getattr(_lib, name)
    fn.restype = res
    fn.argtypes = args
    return fn


_sig("lbx_last_error", C.c_char_p, [])
_sig("lbx_version", C.c_int, [])
_sig("lbx_system_declare", C.c_int, [C.POINTER(SystemDesc), C.POINTER(_P)])
_sig("lbx_system_info", C.c_int, [_P, _I, _I, _I])
_sig("lbx_component_name", C.c_char_p, [_P, C.c_int])
_sig("lbx_system_destroy", None, [_P])
_sig("lbx_scheme_derive", C.c_int, [_P, C.POINTER(SchemeDesc), C.POINTER(_P)])
_sig("lbx_scheme_info", C.c_int, [_P, _D, _D, _D, _D, _I])
_sig("lbx_scheme_destroy", None, [_P])
_sig("lbx_lattice_velocities", C.c_int, [C.c_int, _I, _I, _D])
_sig("lbx_init", C.c_int, [_P, _P, C.c_int, _P, _P, _P, C.POINTER(_P)])
_sig("lbx_state_buffer_bytes", C.c_size_t, [_P])
_sig("lbx_step", C.c_int, [_P, C.c_int64])
_sig("lbx_state_use_graph", C.c_int, [_P, C.c_int])
_sig("lbx_state_set_block", C.c_int, [_P, C.c_int])
_sig("lbx_state_set_staging", C.c_int, [_P, C.c_int])
_sig("lbx_state_set_wait_limit", C.c_int, [_P, C.c_uint64])
_sig("lbx_state_tune", C.c_int, [_P, C.c_int, _I, _I, _D])
_sig("lbx_moments", C.c_int, [_P, _P, C.c_int])
_sig("lbx_conserved_sums", C.c_int, [_P, _D])
_sig("lbx_error_norms", C.c_int, [_P, _P, C.c_int, _D, _D])
_sig("lbx_check_finite", C.c_int, [_P, _I])
_sig("lbx_subchar_check", C.c_int, [_P, _D, _D, _D, _I])
_sig("lbx_get_populations", C.c_int, [_P, _P])
_sig("lbx_set_populations", C.c_int, [_P, _P])
_sig("lbx_state_time", C.c_int, [_P, C.POINTER(C.c_int64), _D])
_sig("lbx_state_populations", _P, [_P])
_sig("lbx_synchronize", C.c_int, [_P])
_sig("lbx_save", C.c_int, [_P, C.c_char_p])
_sig("lbx_load", C.c_int, [_P, C.c_char_p])
_sig("lbx_state_destroy", None, [_P])
_sig("lbx_probe_peaks", C.c_int, [C.c_size_t, _P, _D, _D, _D])
_sig("lbx_conserved_sums_static", C.c_int, [_P, _P, _P, C.c_int, _P])
_sig("lbx_halo_bytes", C.c_size_t, [_P])
_sig("lbx_halo_pack", C.c_int, [_P, _P, _P])
_sig("lbx_halo_unpack", C.c_int, [_P, _P, _P])
_sig("lbx_halo_pack_next", C.c_int, [_P, _P, _P, _P])
_sig("lbx_halo_unpack_next", C.c_int, [_P, _P, _P, _P])
_sig("lbx_step_planes", C.c_int, [_P, C.c_int64, C.c_int64, _P])
_sig("lbx_step_commit", C.c_int, [_P])
_sig("lbx_state_scales", C.c_int, [_P, _D])
_sig("lbx_error_stats", C.c_int, [_P, _P, C.c_int, _D])
_sig("lbx_adjoint", C.c_int, [_P, _P, C.c_int64, C.c_int, _P, _P, _D, _P, _D])
_sig("lbx_adjoint_timings", C.c_int, [_D])
_sig("lbx_adjoint_lam_bytes", C.c_size_t, [_P])
_sig("lbx_adjoint_halo_bytes", C.c_size_t, [_P])
_sig("lbx_adjoint_checkpoint", C.c_int, [_P, _P])
_sig("lbx_adjoint_restore", C.c_int, [_P, _P, C.c_int64])
_sig("lbx_adjoint_seed", C.c_int, [_P, _P, _P, _D])
_sig("lbx_adjoint_step", C.c_int, [_P, _P, _P, _P, _P])
_sig("lbx_adjoint_halo_pack", C.c_int, [_P, _P, _P, _P])
_sig("lbx_adjoint_halo_unpack", C.c_int, [_P, _P, _P, _P])
_sig("lbx_adjoint_finish", C.c_int, [_P, _P, _P, _P, _P, _D])
STATIC_REDUCE_MAX_BLOCKS = 512


def lib():
    """The loaded ctypes library (for callers that need a raw entry point)."""
    return _lib


def check(rc):
    if rc != 0:
        raise LbxError(rc, _lib.lbx_last_error().decode())


def _dbl(n):
    return (C.c_double * n)()


def _host_f64(a):
    """Contiguous float64 numpy view of a CPU tensor or array (kept alive by caller)."""
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def _side(stream):
    """A stream argument of the calls where NULL means the state's own stream."""
    return None if stream is None else _stream_handle(stream)


def _stream_handle(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def lattice_velocities(lattice):
    """(c [q, 3] int, w [q] float64) in the library's population order."""
    q = C.c_int()
    check(_lib.lbx_lattice_velocities(lattice, C.byref(q), None, None))
    c = (C.c_int * (3 * q.value))()
    w = _dbl(q.value)
    check(_lib.lbx_lattice_velocities(lattice, C.byref(q), c, w))
    return np.array(c[:], dtype=np.int64).reshape(q.value, 3), np.array(w[:])


def probe_peaks(nbytes=4 << 30, stream=None, copy=True, fp64=True, fp32=True):
    g, d, s = C.c_double(), C.c_double(), C.c_double()
    check(_lib.lbx_probe_peaks(nbytes, _stream_handle(stream), C.byref(g) if copy else None,
                               C.byref(d) if fp64 else None, C.byref(s) if fp32 else None))
    return {"copy_gbs": g.value if copy else None, "fp64_gflops": d.value if fp64 else None,
            "fp32_gflops": s.value if fp32 else None}


class System:
    """lbx_system_declare: a system family with physical parameters and background Q0."""

    def __init__(self, family, params=(), Q0=()):
        d = SystemDesc()
        d.family = family
        for i, v in enumerate(params):
            d.params[i] = float(v)
        for i, v in enumerate(Q0):
            d.Q0[i] = float(v)
        h = _P()
        check(_lib.lbx_system_declare(C.byref(d), C.byref(h)))
        self._h = h
        K, nc, dim = C.c_int(), C.c_int(), C.c_int()
        check(_lib.lbx_system_info(h, C.byref(K), C.byref(nc), C.byref(dim)))
        self.K, self.n_cons, self.dim = K.value, nc.value, dim.value
        self.names = [_lib.lbx_component_name(h, k).decode() for k in range(self.K)]

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.lbx_system_destroy(self._h)
            self._h = None


class Scheme:
    """lbx_scheme_derive: lattice, extents, refinement law and relaxation slots."""

    def __init__(self, system: System, lattice, extent, scaling, f, tau_lb=0.0, tau_R=0.0,
                 g_tau=0.0, precision=FP64, mms=MMS_NONE, mms_amp=0.0,
                 allow_subchar_violation=False, mms_modes=None, mms_mean=None, mms_conserved_only=False,
                 prescribed=PRESCRIBED_NONE, prescribed_params=(), streaming=STREAM_TWO_BUFFERS,
                 slab_origin=0, slab_planes_global=0, fp16_scales=None):
        """mms_modes: sequence of (p, (kx, ky[, kz]), amp, phase, sigma, omega, psi) for
        MMS_FOURIER; mms_mean: the primitives' means; prescribed, prescribed_params: the
        HCNSF coefficient fields (lbx_prescribed); streaming: STREAM_TWO_BUFFERS or
        STREAM_IN_PLACE (one population buffer, lbx_streaming); slab_origin,
        slab_planes_global: this scheme is the slab of a larger grid starting at that
        global plane of the last axis (extent = the slab's own); fp16_scales: the K storage
        scales of FP16_SCALED instead of the ones derived at init."""
        d = SchemeDesc()
        d.lattice = lattice
        ext = list(extent) + [1] * (3 - len(extent))
        for i in range(3):
            d.extent[i] = int(ext[i])
        d.scaling, d.f, d.tau_lb, d.tau_R, d.g_tau = scaling, float(f), float(tau_lb), float(tau_R), float(g_tau)
        d.precision, d.mms, d.mms_amp = precision, mms, float(mms_amp)
        d.allow_subchar_violation = int(bool(allow_subchar_violation))
        table = None
        if mms_modes is not None:
            table = (MmsMode * len(mms_modes))()
            for m, (pi, k, amp, phase, sigma, omega, psi) in enumerate(mms_modes):
                kk = list(k) + [0] * (3 - len(k))
                table[m].p = int(pi)
                for i in range(3):
                    table[m].k[i] = int(kk[i])
                table[m].amp, table[m].phase, table[m].sigma = float(amp), float(phase), float(sigma)
                table[m].omega, table[m].psi = float(omega), float(psi)
            d.mms_modes = C.cast(table, C.POINTER(MmsMode))
            d.mms_n_modes = len(mms_modes)
        for i, v in enumerate(mms_mean or []):
            d.mms_mean[i] = float(v)
        d.mms_conserved_only = int(bool(mms_conserved_only))
        d.prescribed = int(prescribed)
        for i, v in enumerate(prescribed_params):
            d.prescribed_params[i] = float(v)
        d.streaming = int(streaming)
        d.slab_origin, d.slab_planes_global = int(slab_origin), int(slab_planes_global)
        for i, v in enumerate(fp16_scales or []):
            d.fp16_scales[i] = float(v)
        h = _P()
        check(_lib.lbx_scheme_derive(system._h, C.byref(d), C.byref(h)))
        self._h = h
        self.system = system
        self.lattice = lattice
        self.precision = precision
        self.extent = tuple(int(e) for e in extent)
        dx, dt, lam = C.c_double(), C.c_double(), C.c_double()
        tau = _dbl(system.K)
        q = C.c_int()
        check(_lib.lbx_scheme_info(h, C.byref(dx), C.byref(dt), C.byref(lam), tau, C.byref(q)))
        self.dx, self.dt, self.lam, self.q = dx.value, dt.value, lam.value, q.value
        self.tau = list(tau[:])
        self.grid = tuple(reversed(self.extent))          # (nz,) ny, nx
        self.buffer_bytes = _lib.lbx_state_buffer_bytes(h)
        self.halo_bytes = _lib.lbx_halo_bytes(h)
        self.adjoint_lam_bytes = _lib.lbx_adjoint_lam_bytes(h)
        self.adjoint_halo_bytes = _lib.lbx_adjoint_halo_bytes(h)
        self.slab_origin, self.slab_planes_global = int(slab_origin), int(slab_planes_global)

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.lbx_scheme_destroy(self._h)
            self._h = None


class State:
    """lbx_init ... lbx_state_destroy.  Q: float64 [K, *grid] (CPU or CUDA tensor, or numpy)."""

    def __init__(self, scheme: Scheme, Q, stream=None, buffers=None):
        self.scheme = scheme
        self.K = scheme.system.K
        self._stream = _stream_handle(stream)
        h = _P()
        bufs = (None, None) if buffers is None else tuple(b.data_ptr() if b is not None else None
                                                          for b in (list(buffers) + [None])[:2])
        self._buffers = buffers
        if isinstance(Q, torch.Tensor) and Q.is_cuda:
            Qc = Q.detach().to(torch.float64).contiguous()
            check(_lib.lbx_init(scheme._h, Qc.data_ptr(), 1, self._stream, bufs[0], bufs[1], C.byref(h)))
        else:
            Qh = _host_f64(Q)
            check(_lib.lbx_init(scheme._h, Qh.ctypes.data, 0, self._stream, bufs[0], bufs[1], C.byref(h)))
        self._h = h

    # -- stepping and diagnostics ----------------------------------------------------
    def step(self, n=1):
        check(_lib.lbx_step(self._h, int(n)))

    def set_block(self, block):
        """Threads per block of staged step kernels (32, 64 or 128); results do not change."""
        check(_lib.lbx_state_set_block(self._h, int(block)))

    def set_staging(self, staging):
        """Staging of the staged step kernels: STAGE_AUTO, STAGE_THREAD, STAGE_LANES2,
        STAGE_BULK or STAGE_PIPE (see lbx_state_set_staging)."""
        check(_lib.lbx_state_set_staging(self._h, int(staging)))

    def set_wait_limit(self, ns):
        """lbx_state_set_wait_limit: limit (ns) of the bulk-staged kernels' bounded wait."""
        check(_lib.lbx_state_set_wait_limit(self._h, int(ns)))

    def tune(self, trials=5):
        """lbx_state_tune: pick the fastest staging and block without changing the state;
        returns {"staging", "block", "ms_per_step"}."""
        sg, blk, ms = C.c_int(), C.c_int(), C.c_double()
        check(_lib.lbx_state_tune(self._h, int(trials), C.byref(sg), C.byref(blk), C.byref(ms)))
        return {"staging": sg.value, "block": blk.value, "ms_per_step": ms.value}

    def use_graph(self, enable=True):
        """Replay lbx_step's launches from captured CUDA graphs (needs a non-default stream)."""
        check(_lib.lbx_state_use_graph(self._h, int(bool(enable))))

    def moments(self, device=False):
        """Q [K, *grid] float64.  device=True returns a CUDA tensor written asynchronously on
        the state's stream (synchronize before reading it from another stream)."""
        shape = (self.K,) + self.scheme.grid
        if device:
            out = torch.empty(shape, dtype=torch.float64, device="cuda")
            check(_lib.lbx_moments(self._h, out.data_ptr(), 1))
            return out
        out = np.empty(shape, dtype=np.float64)
        check(_lib.lbx_moments(self._h, out.ctypes.data, 0))
        return torch.from_numpy(out)

    def moments_into(self, out):
        """lbx_moments into a caller-owned float64 tensor [K, *grid]: CUDA (asynchronous on the
        state's stream) or host memory, best page-locked (synchronous)."""
        shape = (self.K,) + self.scheme.grid
        if not (out.dtype == torch.float64 and tuple(out.shape) == shape and out.is_contiguous()):
            raise ValueError(f"moments_into needs a contiguous float64 tensor of shape {shape}")
        check(_lib.lbx_moments(self._h, out.data_ptr(), 1 if out.is_cuda else 0))
        return out

    def halo_pack(self, to_upper, to_lower):
        """lbx_halo_pack into two CUDA uint8 tensors of scheme.halo_bytes bytes."""
        check(_lib.lbx_halo_pack(self._h, to_upper.data_ptr(), to_lower.data_ptr()))

    def step_planes(self, plane0, nplanes, stream=None):
        """lbx_step_planes: planes [plane0, plane0 + nplanes) of the next step (stream None:
        the state's)."""
        check(_lib.lbx_step_planes(self._h, int(plane0), int(nplanes), _side(stream)))

    def step_commit(self):
        check(_lib.lbx_step_commit(self._h))

    def halo_pack_next(self, to_upper, to_lower, stream=None):
        check(_lib.lbx_halo_pack_next(self._h, to_upper.data_ptr(), to_lower.data_ptr(), _side(stream)))

    def halo_unpack_next(self, from_lower, from_upper, stream=None):
        check(_lib.lbx_halo_unpack_next(self._h, from_lower.data_ptr(), from_upper.data_ptr(), _side(stream)))

    def halo_unpack(self, from_lower, from_upper):
        """lbx_halo_unpack from the neighbours' face buffers (CUDA tensors)."""
        check(_lib.lbx_halo_unpack(self._h, from_lower.data_ptr(), from_upper.data_ptr()))

    def scales(self):
        s = _dbl(self.K)
        check(_lib.lbx_state_scales(self._h, s))
        return np.array(s[:])

    def error_stats(self, Q_ref):
        """lbx_error_stats: [K, 4] float64 (sum e^2, sum ref^2, max|e|, max|ref|)."""
        out = _dbl(4 * self.K)
        if isinstance(Q_ref, torch.Tensor) and Q_ref.is_cuda:
            R = Q_ref.detach().to(torch.float64).contiguous()
            check(_lib.lbx_error_stats(self._h, R.data_ptr(), 1, out))
        else:
            R = _host_f64(Q_ref)
            check(_lib.lbx_error_stats(self._h, R.ctypes.data, 0, out))
        return np.array(out[:]).reshape(self.K, 4)

    def conserved_sums(self):
        s = _dbl(self.K)
        check(_lib.lbx_conserved_sums(self._h, s))
        return np.array(s[:])

    def error_norms(self, Q_ref):
        l2, li = _dbl(self.K), _dbl(self.K)
        if isinstance(Q_ref, torch.Tensor) and Q_ref.is_cuda:
            R = Q_ref.detach().to(torch.float64).contiguous()
            check(_lib.lbx_error_norms(self._h, R.data_ptr(), 1, l2, li))
        else:
            R = _host_f64(Q_ref)
            check(_lib.lbx_error_norms(self._h, R.ctypes.data, 0, l2, li))
        return np.array(l2[:]), np.array(li[:])

    def check_finite(self):
        v = C.c_int()
        check(_lib.lbx_check_finite(self._h, C.byref(v)))
        return bool(v.value)

    def subchar_check(self):
        ms, bc, bm, ok = C.c_double(), C.c_double(), C.c_double(), C.c_int()
        check(_lib.lbx_subchar_check(self._h, C.byref(ms), C.byref(bc), C.byref(bm), C.byref(ok)))
        return {"max_speed": ms.value, "bound_cs": bc.value, "bound_monotone": bm.value, "ok": bool(ok.value)}

    def get_populations(self):
        shape = (self.K, self.scheme.q) + self.scheme.grid
        out = np.empty(shape, dtype=np.float64)
        check(_lib.lbx_get_populations(self._h, out.ctypes.data))
        return torch.from_numpy(out)

    def set_populations(self, f):
        fh = _host_f64(f)
        check(_lib.lbx_set_populations(self._h, fh.ctypes.data))

    @property
    def time(self):
        s, t = C.c_int64(), C.c_double()
        check(_lib.lbx_state_time(self._h, C.byref(s), C.byref(t)))
        return s.value, t.value

    def populations_ptr(self):
        return _lib.lbx_state_populations(self._h)

    # step-wise adjoint (include/lbx.h): device tensors throughout
    def adjoint_checkpoint(self, dst):
        """lbx_adjoint_checkpoint: the current populations' bytes into a uint8 CUDA tensor."""
        check(_lib.lbx_adjoint_checkpoint(self._h, dst.data_ptr()))

    def adjoint_restore(self, src, step):
        check(_lib.lbx_adjoint_restore(self._h, src.data_ptr(), int(step)))

    def adjoint_seed(self, rho_target, lam):
        """lbx_adjoint_seed: returns this state's misfit J; rho_target float64 CUDA [cells]."""
        J = C.c_double()
        check(_lib.lbx_adjoint_seed(self._h, rho_target.data_ptr(), lam.data_ptr(), C.byref(J)))
        return J.value

    def adjoint_step(self, An, lam_next, lam_out, tau_acc):
        An_ptr = An if isinstance(An, int) else An.data_ptr()
        check(_lib.lbx_adjoint_step(self._h, An_ptr, lam_next.data_ptr(), lam_out.data_ptr(), tau_acc.data_ptr()))

    def adjoint_halo_pack(self, lam, face_upper, face_lower):
        check(_lib.lbx_adjoint_halo_pack(self._h, lam.data_ptr(), face_upper.data_ptr(), face_lower.data_ptr()))

    def adjoint_halo_unpack(self, lam, face_upper, face_lower):
        check(_lib.lbx_adjoint_halo_unpack(self._h, lam.data_ptr(), face_upper.data_ptr(), face_lower.data_ptr()))

    def adjoint_finish(self, lam0, Q_init, dJ_dQ0, tau_acc):
        """lbx_adjoint_finish: dJ/dQ_init into dJ_dQ0 (float64 CUDA [K, cells]); returns this
        state's share of dJ/dtau."""
        gt = C.c_double()
        check(_lib.lbx_adjoint_finish(self._h, lam0.data_ptr(), Q_init.data_ptr(), dJ_dQ0.data_ptr(),
                                      tau_acc.data_ptr(), C.byref(gt)))
        return gt.value

    def synchronize(self):
        check(_lib.lbx_synchronize(self._h))

    def save(self, path):
        check(_lib.lbx_save(self._h, str(path).encode()))

    def load(self, path):
        check(_lib.lbx_load(self._h, str(path).encode()))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.lbx_state_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


# --------------------------------------------------------------------------- batches
class BatchConfig(C.Structure):
    _fields_ = [("block", C.c_int), ("ctas_per_sm", C.c_int), ("steps_per_launch", C.c_int),
                ("use_graph", C.c_int)]


_sig("lbx_batch_create", C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(_P), _P, C.POINTER(_P)])
_sig("lbx_batch_info", C.c_int, [_P, _I, C.POINTER(C.c_int64), C.POINTER(C.c_size_t)])
_sig("lbx_batch_step", C.c_int, [_P, C.c_int64])
_sig("lbx_batch_check_finite", C.c_int, [_P, _I])
_sig("lbx_batch_synchronize", C.c_int, [_P])
_sig("lbx_batch_moments", C.c_int, [_P, C.c_int, _P])
_sig("lbx_batch_get_config", C.c_int, [_P, C.POINTER(BatchConfig)])
_sig("lbx_batch_set_config", C.c_int, [_P, C.POINTER(BatchConfig)])
_sig("lbx_batch_tune", C.c_int, [_P, C.c_int, C.c_char_p, C.c_size_t])
_sig("lbx_batch_destroy", None, [_P])


class Batch:
    """lbx_batch_create ... lbx_batch_destroy: independent 2D grids advanced together."""

    def __init__(self, schemes, fields, stream=None):
        self.schemes = list(schemes)
        n = len(self.schemes)
        arr = (_P * n)(*[s._h for s in self.schemes])
        host = [_host_f64(Q) for Q in fields]
        qp = (_P * n)(*[h.ctypes.data for h in host])
        h = _P()
        check(_lib.lbx_batch_create(arr, n, qp, None if stream is None else _stream_handle(stream), C.byref(h)))
        self._h = h
        nn, cells, nbytes = C.c_int(), C.c_int64(), C.c_size_t()
        check(_lib.lbx_batch_info(h, C.byref(nn), C.byref(cells), C.byref(nbytes)))
        self.n, self.total_cells, self.buffer_bytes = nn.value, cells.value, nbytes.value

    def step(self, n=1):
        check(_lib.lbx_batch_step(self._h, int(n)))

    def synchronize(self):
        check(_lib.lbx_batch_synchronize(self._h))

    def check_finite(self):
        """Per instance: True when all its populations are finite (lbx_batch_check_finite)."""
        out = (C.c_int * self.n)()
        check(_lib.lbx_batch_check_finite(self._h, out))
        return [bool(v) for v in out]

    def moments(self, j):
        s = self.schemes[j]
        out = np.empty((s.system.K,) + s.grid, dtype=np.float64)
        check(_lib.lbx_batch_moments(self._h, j, out.ctypes.data))
        return torch.from_numpy(out)

    @property
    def config(self):
        c = BatchConfig()
        check(_lib.lbx_batch_get_config(self._h, C.byref(c)))
        return {"block": c.block, "ctas_per_sm": c.ctas_per_sm, "steps_per_launch": c.steps_per_launch,
                "use_graph": bool(c.use_graph)}

    def set_config(self, block=None, ctas_per_sm=None, use_graph=None, steps_per_launch=None):
        cur = self.config
        c = BatchConfig(block or cur["block"], ctas_per_sm or cur["ctas_per_sm"],
                        steps_per_launch or cur["steps_per_launch"],
                        int(cur["use_graph"] if use_graph is None else use_graph))
        check(_lib.lbx_batch_set_config(self._h, C.byref(c)))

    def set_wait_limit(self, ns):
        """lbx_state_set_wait_limit: limit (ns) of the bulk-staged kernels' bounded wait."""
        check(_lib.lbx_state_set_wait_limit(self._h, int(ns)))

    def tune(self, trials=5):
        buf = C.create_string_buffer(1 << 15)
        check(_lib.lbx_batch_tune(self._h, int(trials), buf, len(buf)))
        import json
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "_h", None):
            _lib.lbx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def adjoint(scheme: Scheme, Q_init, n_steps, ckpt_every, rho_target, stream=None):
    """lbx_adjoint: (J, dJ/dQ_init [K, *grid] float64 tensor, dJ/dtau)."""
    Qh = _host_f64(Q_init)
    th = _host_f64(rho_target)
    J, gt = C.c_double(), C.c_double()
    g = np.empty((scheme.system.K,) + scheme.grid, dtype=np.float64)
    check(_lib.lbx_adjoint(scheme._h, Qh.ctypes.data, int(n_steps), int(ckpt_every), th.ctypes.data,
                           _stream_handle(stream), C.byref(J), g.ctypes.data, C.byref(gt)))
    return J.value, torch.from_numpy(g), gt.value


def adjoint_timings():
    """lbx_adjoint_timings: device ms of the last adjoint's forward sweep, recomputation,
    reverse steps and the rest, as a dict."""
    ms = _dbl(4)
    check(_lib.lbx_adjoint_timings(ms))
    return {"forward_ms": ms[0], "recompute_ms": ms[1], "reverse_ms": ms[2], "other_ms": ms[3]}
