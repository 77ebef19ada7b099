"""Thin ctypes binding of include/qtt.h (argument marshalling only).

Every operation runs in the CUDA kernels of libqtt.so; this module converts
NumPy arrays / torch tensors to the plain pointers and sizes of the C-ABI and
raises `QTTError` on a negative status.  There is no fallback: importing it
fails loudly when the shared library has not been built, and creating a
context fails without an sm_103 device.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqtt.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libqtt.so is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = C.CDLL(LIB_PATH)

# Handles still alive when the interpreter shuts down are left to the
# process exit: destroying them after the CUDA runtime has torn down its
# contexts would touch freed driver state.
_ALIVE = [True]
atexit.register(lambda: _ALIVE.__setitem__(0, False))

C128, C64 = 0, 1
PREC_F64, PREC_F32, PREC_TC32, PREC_TF32S = 0, 1, 2, 3
_NP = {C128: np.complex128, C64: np.complex64}


class QTTError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = _lib.qtt_status_string(status).decode()
        super().__init__("%s failed: %s (%d)" % (what, msg, status))


class Complex(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class RoundInfo(C.Structure):
    _fields_ = [("norm", C.c_double), ("delta", C.c_double), ("tail", C.c_double), ("err", C.c_double),
                ("capped", C.c_int32), ("max_rank_out", C.c_int32)]


class RVE(C.Structure):
    _fields_ = [("ncomp", C.c_int32), ("nbits", C.c_int32), ("indicator", C.POINTER(C.c_double)),
                ("k1", C.c_double), ("k2", C.c_double), ("lam1", C.c_double), ("mu1", C.c_double),
                ("lam2", C.c_double), ("mu2", C.c_double), ("interleaved", C.c_int32),
                ("nbits_dim", C.c_int32 * 3), ("boxes", C.POINTER(C.c_double)), ("nboxes", C.c_int32),
                ("op_cross", C.c_int32), ("ellipsoids", C.POINTER(C.c_double)), ("nellipsoids", C.c_int32)]


class CrossFn(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nbits_dim", C.c_int32 * 3), ("interleaved", C.c_int32),
                ("ncomp", C.c_int32), ("k0", C.c_double), ("lam0", C.c_double), ("mu0", C.c_double),
                ("boxes", C.POINTER(C.c_double)), ("nboxes", C.c_int32),
                ("ellipsoids", C.POINTER(C.c_double)), ("nellipsoids", C.c_int32)]


class CrossInfo(C.Structure):
    _fields_ = [("half_sweeps", C.c_int32), ("evaluations", C.c_int64), ("rel_change", C.c_double),
                ("max_rank", C.c_int32)]


CROSS_GREEN, CROSS_BOXES, CROSS_ELLIPSOIDS = 1, 2, 3


class AmenInfo(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("dx", C.c_double)]


class Boxes:
    """A phase geometry without a dense image: a union of axis-aligned boxes
    (rows cx, cy, cz, hx, hy, hz in unit-cell coordinates, periodic) on a grid
    of `shape` = (Nx, Ny, Nz) voxels (powers of two).  The library samples it
    by TT-cross, so the grid may go up to 2^20 voxels per side."""

    def __init__(self, boxes, shape):
        self.boxes = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64).reshape(-1, 6))
        self.shape = tuple(int(n) for n in shape)
        nb = [int(round(np.log2(n))) for n in self.shape]
        if len(nb) != 3 or any((1 << b) != n for b, n in zip(nb, self.shape)):
            raise ValueError("grid sizes must be powers of two, got %s" % (self.shape,))
        self.nbits = nb


class Ellipsoids:
    """A phase geometry without a dense image: a union of ellipsoids (rows of
    15: centre, semi-axes (+inf for a fibre), rotation row-major; see
    inputs.ellipsoids_value) on a grid of `shape` = (Nx, Ny, Nz) voxels
    (powers of two), sampled by TT-cross like Boxes."""

    def __init__(self, rows, shape):
        self.rows = np.ascontiguousarray(np.asarray(rows, dtype=np.float64).reshape(-1, 15))
        self.shape = tuple(int(n) for n in shape)
        nb = [int(round(np.log2(n))) for n in self.shape]
        if len(nb) != 3 or any((1 << b) != n for b, n in zip(nb, self.shape)):
            raise ValueError("grid sizes must be powers of two, got %s" % (self.shape,))
        self.nbits = nb


def _grid_bits(ind):
    """Bits per dimension of an (Nx, Ny, Nz) phase image (powers of two; a
    dimension of one voxel has 0 bits: the plane problem)."""
    if ind.ndim != 3:
        raise ValueError("the phase indicator must be (Nx, Ny, Nz)")
    nb = [int(round(np.log2(n))) for n in ind.shape]
    if any((1 << b) != n for b, n in zip(nb, ind.shape)):
        raise ValueError("grid sizes must be powers of two, got %s" % (ind.shape,))
    return nb


class MSOpts(C.Structure):
    _fields_ = [("prec", C.c_int), ("eps", C.c_double), ("op_tol", C.c_double), ("max_iter", C.c_int32),
                ("oversample", C.c_int32), ("load_mask", C.c_int32), ("min_iter", C.c_int32),
                ("seed", C.c_uint64), ("predictor", C.c_void_p), ("trace", C.POINTER(C.c_float)),
                ("trace_cap", C.c_int64), ("green_amen", C.c_int32), ("strain", C.POINTER(C.c_void_p)),
                ("lc_workers", C.c_int32), ("warm_iter", C.c_int32)]


class MSReport(C.Structure):
    _fields_ = [("iterations", C.c_int32 * 6), ("residual", C.c_double * 6), ("sigma_imag_max", C.c_double),
                ("max_rank_seen", C.c_int32), ("setup_ms", C.c_double), ("iterate_ms", C.c_double),
                ("kernel_launches", C.c_int64), ("trace_len", C.c_int64), ("sketch_width_sum", C.c_int64),
                ("fallbacks", C.c_int32), ("green_rank", C.c_int32), ("phase_rank", C.c_int32),
                ("fp64_residuals", C.c_int32), ("timed_ms", C.c_double), ("timed_iter", C.c_int32),
                ("timed_launches", C.c_int64), ("post_checks", C.c_int32), ("svd_fallbacks", C.c_int32),
                ("post_err_max", C.c_double)]


MLP_FEATURES = 10


_P = C.c_void_p
_I32P = C.POINTER(C.c_int32)


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("qtt_status_string", C.c_char_p, [C.c_int])
_sig("qtt_ctx_create", C.c_int, [C.c_int, _P, C.POINTER(_P)])
_sig("qtt_ctx_destroy", None, [_P])
_sig("qtt_ctx_sync", C.c_int, [_P])
_sig("qtt_ctx_launch_count", C.c_int64, [_P])
_sig("qtt_ctx_fail_alloc_after", C.c_int, [_P, C.c_int64])
_sig("qtt_measure_peak", C.c_int, [_P, C.c_int, C.POINTER(C.c_double)])
_sig("qtt_ctx_profile", C.c_int, [_P, C.c_int])
_sig("qtt_ctx_profile_read", C.c_int, [_P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                        C.POINTER(C.c_double), C.POINTER(C.c_double)])
_sig("qtt_ctx_profile_shapes", C.c_int, [_P, C.c_int, C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int64)])
_sig("qtt_tt_create", C.c_int, [_P, C.c_int, _I32P, _I32P, C.c_int, C.POINTER(_P)])
_sig("qtt_tt_destroy", None, [_P])
_sig("qtt_tt_ncores", C.c_int, [_P])
_sig("qtt_tt_ranks", C.c_int, [_P, _I32P])
_sig("qtt_tt_modes", C.c_int, [_P, _I32P])
_sig("qtt_tt_dtype", C.c_int, [_P])
_sig("qtt_tt_core_ptr", _P, [_P, C.c_int])
_sig("qtt_tt_from_host", C.c_int, [_P, C.c_int, _P])
_sig("qtt_tt_to_host", C.c_int, [_P, C.c_int, _P])
_sig("qtt_tt_from_device", C.c_int, [_P, C.c_int, _P])
_sig("qtt_tt_convert", C.c_int, [_P, _P, C.c_int, C.POINTER(_P)])
_sig("qtt_mpo_create", C.c_int, [_P, C.c_int, _I32P, _I32P, _I32P, C.c_int, C.POINTER(_P)])
_sig("qtt_mpo_destroy", None, [_P])
_sig("qtt_mpo_ranks", C.c_int, [_P, _I32P])
_sig("qtt_mpo_from_host", C.c_int, [_P, C.c_int, _P])
_sig("qtt_mpo_to_host", C.c_int, [_P, C.c_int, _P])
_sig("tt_add", C.c_int, [_P, Complex, _P, Complex, _P, C.POINTER(_P)])
_sig("tt_hadamard", C.c_int, [_P, _P, _P, C.POINTER(_P)])
_sig("tt_mpo_apply", C.c_int, [_P, _P, _P, C.POINTER(_P)])
_sig("tt_round", C.c_int, [_P, _P, C.c_double, C.c_int, C.c_int, C.POINTER(RoundInfo), C.POINTER(_P)])
_sig("tt_round_polar", C.c_int, [_P, _P, C.c_double, C.c_int, C.POINTER(RoundInfo), C.POINTER(_P)])
_sig("tt_round_batch", C.c_int, [_P, C.c_int, C.POINTER(_P), C.c_double, C.c_int, C.c_int, C.POINTER(RoundInfo),
                                 C.POINTER(_P)])
_sig("tt_round_sketched", C.c_int, [_P, C.c_int, C.POINTER(Complex), C.POINTER(_P), C.POINTER(_P), _P,
                                    C.c_double, C.c_int, C.c_int, C.POINTER(RoundInfo), C.POINTER(_P)])
_sig("tt_dot", C.c_int, [_P, _P, _P, C.POINTER(C.c_double)])
_sig("tt_dot_structured", C.c_int, [_P, C.c_int, C.POINTER(Complex), C.POINTER(_P), C.POINTER(_P), _P,
                                    C.POINTER(C.c_double)])
_sig("tt_norm", C.c_int, [_P, _P, C.POINTER(C.c_double)])
_sig("tt_from_dense", C.c_int, [_P, C.c_int, _I32P, _P, C.c_double, C.c_int, C.POINTER(_P)])
_sig("qtt_qft_mpo", C.c_int, [_P, C.c_int, C.c_int, C.c_double, C.POINTER(_P)])
_sig("qtt_mpo_diag", C.c_int, [_P, _P, C.POINTER(_P)])
_sig("qtt_cgemm", C.c_int, [_P, C.c_int64, C.c_int64, C.c_int64, _P, _P, _P, C.c_int])
_sig("qtt_cgemm_noalloc", C.c_int, [_P, C.c_int64, C.c_int64, C.c_int64, _P, _P, _P])
_sig("qtt_mpo_convert", C.c_int, [_P, _P, C.c_int, C.POINTER(_P)])
_sig("ms_homogenize_batch", C.c_int, [_P, C.c_int, C.POINTER(RVE), C.POINTER(C.c_double), C.c_double, C.c_int,
                                      C.POINTER(MSOpts), C.c_int, C.POINTER(C.c_double), C.POINTER(MSReport)])
_sig("qtt_mlp_create", C.c_int, [_P, C.c_int, C.c_uint64, C.POINTER(_P)])
_sig("qtt_mlp_destroy", None, [_P])
_sig("qtt_mlp_param_count", C.c_int64, [_P])
_sig("qtt_mlp_set_params", C.c_int, [_P, C.POINTER(C.c_float), C.c_int64])
_sig("qtt_mlp_get_params", C.c_int, [_P, C.POINTER(C.c_float), C.c_int64])
_sig("qtt_mlp_forward", C.c_int, [_P, C.POINTER(C.c_float), C.c_int64, C.POINTER(C.c_float)])
_sig("qtt_mlp_train_step", C.c_int, [_P, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int64, C.c_float,
                                     C.c_float, C.POINTER(C.c_double), C.POINTER(C.c_float)])
_sig("qtt_site_order", C.c_int, [_I32P, C.c_int32, _I32P, _I32P])
_sig("tt_contract_voxels", C.c_int, [_P, _P, _I32P, C.c_int32, _P])
_sig("tt_amen_mv", C.c_int, [_P, _P, _P, _P, C.c_double, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(_P),
                            C.POINTER(AmenInfo)])
_sig("tt_cross", C.c_int, [_P, C.POINTER(CrossFn), C.c_double, C.c_int32, C.c_int32, C.c_int32, C.c_uint64,
                          C.POINTER(_P), C.POINTER(CrossInfo)])
_sig("ms_homogenize", C.c_int, [_P, C.POINTER(RVE), C.POINTER(C.c_double), C.c_double, C.c_int,
                                C.POINTER(MSOpts), C.POINTER(C.c_double), C.POINTER(MSReport)])
_sig("ms_setup", C.c_int, [_P, C.POINTER(RVE), C.POINTER(C.c_double), C.c_double, C.c_int, C.POINTER(_P)])
_sig("ms_homogenize_ops", C.c_int, [_P, _P, C.c_double, C.c_int, C.POINTER(MSOpts), C.POINTER(C.c_double),
                                    C.POINTER(MSReport)])
_sig("ms_ops_destroy", None, [_P])
_sig("ms_ops_ranks", C.c_int, [_P, _I32P, _I32P])

EXPORTED = ["qtt_status_string", "qtt_ctx_create", "qtt_ctx_destroy", "qtt_ctx_sync", "qtt_ctx_launch_count",
            "qtt_ctx_fail_alloc_after", "qtt_measure_peak",
            "qtt_ctx_profile", "qtt_ctx_profile_read", "qtt_ctx_profile_shapes",
            "qtt_tt_create", "qtt_tt_destroy", "qtt_tt_ncores", "qtt_tt_ranks", "qtt_tt_modes", "qtt_tt_dtype",
            "qtt_tt_core_ptr", "qtt_tt_from_host", "qtt_tt_to_host", "qtt_tt_from_device", "qtt_tt_convert",
            "qtt_mpo_create", "qtt_mpo_destroy", "qtt_mpo_ranks", "qtt_mpo_from_host", "qtt_mpo_to_host",
            "tt_add", "tt_hadamard", "tt_mpo_apply", "tt_round", "tt_round_polar", "tt_round_batch", "tt_round_sketched", "tt_dot", "tt_dot_structured", "tt_norm",
            "tt_from_dense", "tt_cross", "tt_amen_mv", "tt_contract_voxels", "qtt_site_order", "qtt_qft_mpo", "qtt_mpo_diag", "qtt_mpo_convert", "ms_homogenize",
            "ms_homogenize_batch", "ms_setup", "ms_homogenize_ops", "ms_ops_destroy", "ms_ops_ranks",
            "qtt_cgemm", "qtt_cgemm_noalloc",
            "qtt_mlp_create", "qtt_mlp_destroy", "qtt_mlp_param_count", "qtt_mlp_set_params",
            "qtt_mlp_get_params", "qtt_mlp_forward", "qtt_mlp_train_step"]


def _check(st, what):
    if st != 0:
        raise QTTError(st, what)


def _i32(seq):
    a = (C.c_int32 * len(seq))(*[int(v) for v in seq])
    return a


class Context:
    """A device context bound to a CUDA stream (torch's current stream by default)."""

    def __init__(self, device: int = 0, stream=None):
        h = _P()
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:  # torch is optional plumbing
                stream = None
        _check(_lib.qtt_ctx_create(int(device), _P(stream) if stream else None, C.byref(h)), "qtt_ctx_create")
        self.h = h
        # Trains, operators and predictors free their device memory on this
        # context's stream, so the context is destroyed only after the last of
        # them: a reference cycle collected in one pass may finalise the
        # context before its children.
        self._children = 0
        self._close_pending = False

    def _adopt(self):
        self._children += 1

    def _release(self):
        self._children -= 1
        if self._children <= 0 and self._close_pending:
            self._destroy()

    def _destroy(self):
        if getattr(self, "h", None) and _ALIVE[0]:
            _lib.qtt_ctx_destroy(self.h)
        self.h = None

    def close(self):
        if getattr(self, "_children", 0) > 0:
            self._close_pending = True
        else:
            self._destroy()

    def __del__(self):
        self.close()

    def sync(self):
        _check(_lib.qtt_ctx_sync(self.h), "qtt_ctx_sync")

    @property
    def launches(self) -> int:
        return int(_lib.qtt_ctx_launch_count(self.h))

    def fail_alloc_after(self, n: int):
        """Test hook: the allocation after `n` more succeed fails (QTT_ERR_OOM); n < 0 turns it off."""
        _check(_lib.qtt_ctx_fail_alloc_after(self.h, int(n)), "qtt_ctx_fail_alloc_after")

    def measure_peak(self, which: str) -> float:
        """Peak of this GPU in TFLOP/s: FMA chains ("fp32", "fp64") or tcgen05
        MMAs from shared memory ("tf32", "bf16")."""
        out = C.c_double()
        _check(_lib.qtt_measure_peak(self.h, {"fp32": 0, "fp64": 1, "tf32": 2, "bf16": 3}[which], C.byref(out)),
               "qtt_measure_peak")
        return float(out.value)

    KERNEL_CLASSES = {"gemm": 0, "qr": 1, "jacobi": 2, "elem": 3}

    def profile(self, enable):
        """True/1: record every launch; 2: only the timed iterations of
        ms_homogenize (report.timed_ms); False/0: off."""
        mode = 2 if enable == 2 else (1 if enable else 0)
        _check(_lib.qtt_ctx_profile(self.h, mode), "qtt_ctx_profile")

    def profile_read(self, kclass: str):
        ms, fl, by = C.c_double(), C.c_double(), C.c_double()
        n = C.c_int64()
        _check(_lib.qtt_ctx_profile_read(self.h, self.KERNEL_CLASSES[kclass], C.byref(ms), C.byref(n), C.byref(fl),
                                         C.byref(by)), "qtt_ctx_profile_read")
        return {"ms": ms.value, "launches": int(n.value), "flops": fl.value, "bytes": by.value}

    def profile_shapes(self, kclass: str, max_rows: int = 64):
        """This context's records of one class grouped by launch shape, by
        decreasing total time: dicts with dims (GEMM M, N, K; QR m, n, 0;
        Jacobi p, q, 0), batch, variant, launches, ms and flops."""
        n = C.c_int64()
        rows = np.zeros((max_rows, 8), dtype=np.float64)
        _check(_lib.qtt_ctx_profile_shapes(self.h, self.KERNEL_CLASSES[kclass],
                                           rows.ctypes.data_as(C.POINTER(C.c_double)), max_rows, C.byref(n)),
               "qtt_ctx_profile_shapes")
        out = []
        for r in rows[:min(max_rows, int(n.value))]:
            out.append({"dims": tuple(int(v) for v in r[:3]), "batch": int(r[3]), "variant": int(r[4]),
                        "launches": int(r[5]), "ms": float(r[6]), "flops": float(r[7])})
        return out


class TT:
    """Handle of a library-owned tensor train."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.h = handle
        ctx._adopt()
        self._adopted = True

    @classmethod
    def from_cores(cls, ctx: Context, cores, dtype=C128):
        cores = [np.ascontiguousarray(c, dtype=_NP[dtype]) for c in cores]
        d = len(cores)
        modes = [c.shape[1] for c in cores]
        ranks = [cores[0].shape[0]] + [c.shape[2] for c in cores]
        h = _P()
        _check(_lib.qtt_tt_create(ctx.h, d, _i32(modes), _i32(ranks), dtype, C.byref(h)), "qtt_tt_create")
        t = cls(ctx, h)
        for k, c in enumerate(cores):
            _check(_lib.qtt_tt_from_host(h, k, c.ctypes.data), "qtt_tt_from_host")
        return t

    def close(self):
        if getattr(self, "h", None) and _ALIVE[0]:
            _lib.qtt_tt_destroy(self.h)
        self.h = None
        if getattr(self, "_adopted", False):
            self._adopted = False
            self.ctx._release()

    def __del__(self):
        self.close()

    @property
    def ncores(self) -> int:
        return int(_lib.qtt_tt_ncores(self.h))

    @property
    def ranks(self):
        r = (C.c_int32 * (self.ncores + 1))()
        _check(_lib.qtt_tt_ranks(self.h, r), "qtt_tt_ranks")
        return list(r)

    @property
    def modes(self):
        m = (C.c_int32 * self.ncores)()
        _check(_lib.qtt_tt_modes(self.h, m), "qtt_tt_modes")
        return list(m)

    @property
    def dtype(self) -> int:
        return int(_lib.qtt_tt_dtype(self.h))

    def cores(self):
        out = []
        r, m = self.ranks, self.modes
        for k in range(self.ncores):
            a = np.empty((r[k], m[k], r[k + 1]), dtype=_NP[self.dtype])
            _check(_lib.qtt_tt_to_host(self.h, k, a.ctypes.data), "qtt_tt_to_host")
            out.append(a)
        return out

    def core_ptr(self, k: int) -> int:
        return int(_lib.qtt_tt_core_ptr(self.h, k))

    def convert(self, dtype):
        h = _P()
        _check(_lib.qtt_tt_convert(self.ctx.h, self.h, dtype, C.byref(h)), "qtt_tt_convert")
        return TT(self.ctx, h)


class MPO:
    def __init__(self, ctx: Context, handle, d: int):
        self.ctx = ctx
        self.h = handle
        self.d = d
        ctx._adopt()
        self._adopted = True

    @classmethod
    def from_cores(cls, ctx: Context, cores, dtype=C128):
        cores = [np.ascontiguousarray(c, dtype=_NP[dtype]) for c in cores]
        d = len(cores)
        mo = [c.shape[1] for c in cores]
        mi = [c.shape[2] for c in cores]
        g = [cores[0].shape[0]] + [c.shape[3] for c in cores]
        h = _P()
        _check(_lib.qtt_mpo_create(ctx.h, d, _i32(mo), _i32(mi), _i32(g), dtype, C.byref(h)), "qtt_mpo_create")
        A = cls(ctx, h, d)
        for k, c in enumerate(cores):
            _check(_lib.qtt_mpo_from_host(h, k, c.ctypes.data), "qtt_mpo_from_host")
        A._shapes = [c.shape for c in cores]
        A._dtype = dtype
        return A

    def close(self):
        if getattr(self, "h", None) and _ALIVE[0]:
            _lib.qtt_mpo_destroy(self.h)
        self.h = None
        if getattr(self, "_adopted", False):
            self._adopted = False
            self.ctx._release()

    def __del__(self):
        self.close()

    @property
    def ranks(self):
        r = (C.c_int32 * (self.d + 1))()
        _check(_lib.qtt_mpo_ranks(self.h, r), "qtt_mpo_ranks")
        return list(r)

    def cores(self, shapes=None, dtype=C128):
        shapes = shapes or self._shapes
        out = []
        for k, s in enumerate(shapes):
            a = np.empty(s, dtype=_NP[dtype])
            _check(_lib.qtt_mpo_to_host(self.h, k, a.ctypes.data), "qtt_mpo_to_host")
            out.append(a)
        return out


def _cx(v) -> Complex:
    v = complex(v)
    return Complex(v.real, v.imag)


def tt_add(ctx: Context, a, x: TT, b, y: TT) -> TT:
    h = _P()
    _check(_lib.tt_add(ctx.h, _cx(a), x.h, _cx(b), y.h, C.byref(h)), "tt_add")
    return TT(ctx, h)


def tt_hadamard(ctx: Context, x: TT, y: TT) -> TT:
    h = _P()
    _check(_lib.tt_hadamard(ctx.h, x.h, y.h, C.byref(h)), "tt_hadamard")
    return TT(ctx, h)


def tt_mpo_apply(ctx: Context, A: MPO, x: TT) -> TT:
    h = _P()
    _check(_lib.tt_mpo_apply(ctx.h, A.h, x.h, C.byref(h)), "tt_mpo_apply")
    return TT(ctx, h)


def site_order(nbits, interleaved: bool = True):
    """(dim, pos) of every spatial site of a 2^nbits grid (host only)."""
    nb = [int(b) for b in nbits]
    n = max(sum(nb), 1)
    dim = (C.c_int32 * n)()
    pos = (C.c_int32 * n)()
    d = _lib.qtt_site_order(_i32(nb), 1 if interleaved else 0, dim, pos)
    if d < 0:
        _check(d, "qtt_site_order")
    return list(dim[:d]), list(pos[:d])


def contract_voxels(ctx: Context, x: TT, nbits, interleaved: bool = True) -> np.ndarray:
    """Algorithm 2's contract(): the full tensor of x (control core first, or
    spatial sites only) as a voxel field (ncomp, Nx, Ny, Nz)."""
    nb = [int(b) for b in nbits]
    ncomp = x.modes[0] if x.ncores == sum(nb) + 1 else 1
    out = np.zeros((ncomp, 1 << nb[0], 1 << nb[1], 1 << nb[2]), dtype=_NP[x.dtype])
    _check(_lib.tt_contract_voxels(ctx.h, x.h, _i32(nb), 1 if interleaved else 0, out.ctypes.data),
           "tt_contract_voxels")
    return out


def tt_amen_mv(ctx: Context, A: MPO, x: TT, eps: float, y0: TT | None = None, kick: int = 4, max_sweeps: int = 20,
               seed: int = 1):
    """y ~ A x by AMEn (never forms A x); returns (TT, AmenInfo)."""
    h = _P()
    info = AmenInfo()
    _check(_lib.tt_amen_mv(ctx.h, A.h, x.h, y0.h if y0 is not None else None, float(eps), int(kick),
                           int(max_sweeps), int(seed), C.byref(h), C.byref(info)), "tt_amen_mv")
    return TT(ctx, h), info


def tt_round(ctx: Context, x: TT, eps: float, max_rank: int = 0, prec=None):
    if prec is None:
        prec = PREC_F64 if x.dtype == C128 else PREC_F32
    h = _P()
    info = RoundInfo()
    _check(_lib.tt_round(ctx.h, x.h, float(eps), int(max_rank), int(prec), C.byref(info), C.byref(h)), "tt_round")
    return TT(ctx, h), info


def tt_round_polar(ctx: Context, x: TT, eps: float, prec=None):
    if prec is None:
        prec = PREC_F64 if x.dtype == C128 else PREC_F32
    h = _P()
    info = RoundInfo()
    _check(_lib.tt_round_polar(ctx.h, x.h, float(eps), int(prec), C.byref(info), C.byref(h)), "tt_round_polar")
    return TT(ctx, h), info


def tt_cross(ctx: Context, kind: str, nbits, eps: float, interleaved: bool = True, ncomp: int = 3,
             k0: float = 1.0, lam0: float = 0.0, mu0: float = 0.0, boxes=None, max_rank: int = 0,
             kick: int | None = None, max_half_sweeps: int = 24, seed: int = 1, ellipsoids=None):
    """TT-cross of the Green operator train (kind "green": modes (ncomp^2,
    2, ...), momentum convention) or of a box / ellipsoid geometry's phase
    indicator (kind "boxes" / "ellipsoids": modes (2, ...), position
    convention) on a grid of 2^nbits[a] voxels per dimension; kick defaults
    to 4 (green) / 8 (geometries), as inside ms_homogenize.  Returns
    (TT, CrossInfo)."""
    if kick is None:
        kick = 4 if kind == "green" else 8
    f = CrossFn()
    f.kind = {"green": CROSS_GREEN, "boxes": CROSS_BOXES, "ellipsoids": CROSS_ELLIPSOIDS}[kind]
    for a in range(3):
        f.nbits_dim[a] = int(nbits[a])
    f.interleaved = 1 if interleaved else 0
    f.ncomp, f.k0, f.lam0, f.mu0 = int(ncomp), float(k0), float(lam0), float(mu0)
    keep = None
    if boxes is not None:
        keep = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64).reshape(-1, 6))
        f.boxes = keep.ctypes.data_as(C.POINTER(C.c_double))
        f.nboxes = keep.shape[0]
    if ellipsoids is not None:
        keep = np.ascontiguousarray(np.asarray(ellipsoids, dtype=np.float64).reshape(-1, 15))
        f.ellipsoids = keep.ctypes.data_as(C.POINTER(C.c_double))
        f.nellipsoids = keep.shape[0]
    h = _P()
    info = CrossInfo()
    _check(_lib.tt_cross(ctx.h, C.byref(f), float(eps), int(max_rank), int(kick), int(max_half_sweeps), int(seed),
                         C.byref(h), C.byref(info)), "tt_cross")
    return TT(ctx, h), info


def tt_round_batch(ctx: Context, xs, eps: float, max_rank: int = 0, prec=None):
    """Round trains of one shape together; returns (list of TT, list of RoundInfo)."""
    xs = list(xs)
    if prec is None:
        prec = PREC_F64 if xs[0].dtype == C128 else PREC_F32
    B = len(xs)
    hin = (_P * B)(*[x.h for x in xs])
    hout = (_P * B)()
    infos = (RoundInfo * B)()
    _check(_lib.tt_round_batch(ctx.h, B, hin, float(eps), int(max_rank), int(prec), infos, hout), "tt_round_batch")
    return [TT(ctx, _P(hout[b])) for b in range(B)], [infos[b] for b in range(B)]


def tt_round_sketched(ctx: Context, terms, sketch: TT, eps: float, max_rank: int = 0, prec=None):
    """terms: list of (coef, MPO or None, TT)."""
    if prec is None:
        prec = PREC_F64 if sketch.dtype == C128 else PREC_F32
    T = len(terms)
    coefs = (Complex * T)(*[_cx(c) for c, _, _ in terms])
    ops = (_P * T)(*[(A.h if A is not None else None) for _, A, _ in terms])
    xs = (_P * T)(*[x.h for _, _, x in terms])
    h = _P()
    info = RoundInfo()
    _check(_lib.tt_round_sketched(ctx.h, T, coefs, ops, xs, sketch.h, float(eps), int(max_rank), int(prec),
                                  C.byref(info), C.byref(h)), "tt_round_sketched")
    return TT(ctx, h), info


def tt_dot(ctx: Context, x: TT, y: TT) -> complex:
    out = (C.c_double * 2)()
    _check(_lib.tt_dot(ctx.h, x.h, y.h, out), "tt_dot")
    return complex(out[0], out[1])


def tt_dot_structured(ctx: Context, terms, y: TT) -> complex:
    """<y, sum_t c_t A_t x_t> for terms (c_t, MPO or None, TT), without forming the sum."""
    T = len(terms)
    coefs = (Complex * T)(*[_cx(c) for c, _, _ in terms])
    ops = (_P * T)(*[(A.h if A is not None else None) for _, A, _ in terms])
    xs = (_P * T)(*[x.h for _, _, x in terms])
    out = (C.c_double * 2)()
    _check(_lib.tt_dot_structured(ctx.h, T, coefs, ops, xs, y.h, out), "tt_dot_structured")
    return complex(out[0], out[1])


def tt_norm(ctx: Context, x: TT) -> float:
    out = C.c_double()
    _check(_lib.tt_norm(ctx.h, x.h, C.byref(out)), "tt_norm")
    return float(out.value)


def tt_from_dense(ctx: Context, dense_device_ptr: int, modes, eps: float, max_rank: int = 0) -> TT:
    """TT-SVD of a complex128 dense tensor already in device memory (e.g. a torch tensor's data_ptr())."""
    h = _P()
    _check(_lib.tt_from_dense(ctx.h, len(modes), _i32(modes), _P(dense_device_ptr), float(eps), int(max_rank),
                              C.byref(h)), "tt_from_dense")
    return TT(ctx, h)


def qtt_qft_mpo(ctx: Context, nbits: int, sign: int = -1, tol: float = 1e-12) -> MPO:
    h = _P()
    _check(_lib.qtt_qft_mpo(ctx.h, int(nbits), int(sign), float(tol), C.byref(h)), "qtt_qft_mpo")
    A = MPO(ctx, h, nbits)
    g = A.ranks
    A._shapes = [(g[k], 2, 2, g[k + 1]) for k in range(nbits)]
    A._dtype = C128
    return A


def qtt_cgemm(ctx: Context, M: int, N: int, K: int, A_ptr: int, B_ptr: int, C_ptr: int, engine: int = 1):
    """C = A B for row-major complex64 device buffers (e.g. torch tensors' data_ptr())."""
    _check(_lib.qtt_cgemm(ctx.h, int(M), int(N), int(K), _P(A_ptr), _P(B_ptr), _P(C_ptr), int(engine)), "qtt_cgemm")


def qtt_cgemm_noalloc(stream: int, M: int, N: int, K: int, A_ptr: int, B_ptr: int, C_ptr: int):
    """Tensor-core C = A B that allocates no device memory (fixed 16 MiB library
    array); for callers that may not allocate.  `stream` is a cudaStream_t value."""
    _check(_lib.qtt_cgemm_noalloc(_P(stream) if stream else None, int(M), int(N), int(K), _P(A_ptr), _P(B_ptr),
                                  _P(C_ptr)), "qtt_cgemm_noalloc")


def qtt_mpo_diag(ctx: Context, x: TT) -> MPO:
    h = _P()
    _check(_lib.qtt_mpo_diag(ctx.h, x.h, C.byref(h)), "qtt_mpo_diag")
    A = MPO(ctx, h, x.ncores)
    r, m = x.ranks, x.modes
    A._shapes = [(r[k], m[k], m[k], r[k + 1]) for k in range(x.ncores)]
    A._dtype = x.dtype
    return A


def qtt_mpo_convert(ctx: Context, A: MPO, dtype) -> MPO:
    h = _P()
    _check(_lib.qtt_mpo_convert(ctx.h, A.h, int(dtype), C.byref(h)), "qtt_mpo_convert")
    B = MPO(ctx, h, A.d)
    B._shapes = getattr(A, "_shapes", None)
    B._dtype = dtype
    return B


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class MLP:
    """The per-bond rank predictor (3 hidden layers of 64, FP16 weights) on the device."""

    def __init__(self, ctx: Context, n_features: int = MLP_FEATURES, seed: int = 0):
        self.ctx = ctx
        h = _P()
        _check(_lib.qtt_mlp_create(ctx.h, int(n_features), int(seed), C.byref(h)), "qtt_mlp_create")
        self.h = h
        ctx._adopt()
        self._adopted = True
        self.n_features = n_features

    def close(self):
        if getattr(self, "h", None) and _ALIVE[0]:
            _lib.qtt_mlp_destroy(self.h)
        self.h = None
        if getattr(self, "_adopted", False):
            self._adopted = False
            self.ctx._release()

    def __del__(self):
        self.close()

    @property
    def param_count(self) -> int:
        return int(_lib.qtt_mlp_param_count(self.h))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.param_count, dtype=np.float32)
        _check(_lib.qtt_mlp_get_params(self.h, _fptr(p), p.size), "qtt_mlp_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(_lib.qtt_mlp_set_params(self.h, _fptr(p), p.size), "qtt_mlp_set_params")

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.empty(X.shape[0], dtype=np.float32)
        _check(_lib.qtt_mlp_forward(self.h, _fptr(X), X.shape[0], _fptr(y)), "qtt_mlp_forward")
        return y

    def train_step(self, X, t, alpha: float = 4.0, lr: float = 1e-3, want_grads: bool = False):
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        loss = C.c_double()
        g = np.empty(self.param_count, dtype=np.float32) if want_grads else None
        _check(_lib.qtt_mlp_train_step(self.h, _fptr(X), _fptr(t), X.shape[0], float(alpha), float(lr),
                                       C.byref(loss), _fptr(g) if g is not None else None), "qtt_mlp_train_step")
        return (loss.value, g) if want_grads else loss.value


def _rve(ind, kind, moduli, interleaved, op_cross=False):
    """qtt_rve for a dense phase image (Nx, Ny, Nz), a Boxes or an Ellipsoids geometry;
    returns (rve, arrays kept alive for the call)."""
    rve = RVE()
    if isinstance(ind, Boxes):
        nb = ind.nbits
        keep = ind.boxes
        rve.boxes = keep.ctypes.data_as(C.POINTER(C.c_double))
        rve.nboxes = keep.shape[0]
    elif isinstance(ind, Ellipsoids):
        nb = ind.nbits
        keep = ind.rows
        rve.ellipsoids = keep.ctypes.data_as(C.POINTER(C.c_double))
        rve.nellipsoids = keep.shape[0]
    else:
        keep = np.ascontiguousarray(ind, dtype=np.float64)
        nb = _grid_bits(keep)
        rve.indicator = keep.ctypes.data_as(C.POINTER(C.c_double))
    rve.nbits = max(nb)
    rve.nbits_dim[0], rve.nbits_dim[1], rve.nbits_dim[2] = nb
    rve.interleaved = 1 if interleaved else 0
    rve.op_cross = 1 if op_cross else 0
    if kind == "scalar":
        rve.ncomp = 3
        rve.k1, rve.k2 = map(float, moduli)
    else:
        rve.ncomp = 6
        rve.lam1, rve.mu1, rve.lam2, rve.mu2 = map(float, moduli)
    return rve, keep


def ms_homogenize_batch(ctx: Context, problems, tol: float, max_rank: int, workers: int = 8, eps: float = 1e-6,
                        op_tol: float = 1e-10, prec: int = PREC_F64, max_iter: int = 100, oversample: int = 8,
                        load_mask: int = 0x3F, interleaved: bool = True, min_iter: int = 1, seed: int = 12345,
                        predictor: "MLP | None" = None):
    """problems: list of (indicator, kind, moduli, C0).  Returns ([C_eff], [report])."""
    n = len(problems)
    rves = (RVE * max(n, 1))()
    keep = []
    C0s = np.zeros((max(n, 1), 36), dtype=np.float64)
    sizes = []
    for i, (ind, kind, moduli, C0) in enumerate(problems):
        r, a = _rve(ind, kind, moduli, interleaved)
        keep.append(a)
        rves[i] = r
        nc = r.ncomp
        C0s[i, :nc * nc] = np.asarray(C0, dtype=np.float64).reshape(-1)
        sizes.append(nc)
    o = MSOpts()
    o.prec, o.eps, o.op_tol, o.max_iter = int(prec), float(eps), float(op_tol), int(max_iter)
    o.oversample, o.load_mask, o.min_iter, o.seed = int(oversample), int(load_mask), int(min_iter), int(seed)
    o.predictor = predictor.h if predictor is not None else None
    o.trace, o.trace_cap = None, 0
    out = np.zeros(sum(s * s for s in sizes) + 1, dtype=np.float64)
    reps = (MSReport * max(n, 1))()
    _check(_lib.ms_homogenize_batch(ctx.h, n, rves, C0s.ctypes.data_as(C.POINTER(C.c_double)), float(tol),
                                    int(max_rank), C.byref(o), int(workers),
                                    out.ctypes.data_as(C.POINTER(C.c_double)), reps), "ms_homogenize_batch")
    res, off = [], 0
    for nc in sizes:
        res.append(out[off:off + nc * nc].reshape(nc, nc).copy())
        off += nc * nc
    return res, [reps[i] for i in range(n)]


class MSOps:
    """The operator trains of one RVE (ms_setup), reusable by many solves."""

    def __init__(self, ctx: Context, handle, ncomp: int, setup_ms: float):
        self.ctx = ctx
        self.h = handle
        self.ncomp = ncomp
        self.setup_ms = setup_ms
        ctx._adopt()
        self._adopted = True

    @property
    def ranks(self):
        g, p = C.c_int32(), C.c_int32()
        _check(_lib.ms_ops_ranks(self.h, C.byref(g), C.byref(p)), "ms_ops_ranks")
        return int(g.value), int(p.value)

    def close(self):
        if getattr(self, "h", None) and _ALIVE[0]:
            _lib.ms_ops_destroy(self.h)
        self.h = None
        if getattr(self, "_adopted", False):
            self._adopted = False
            self.ctx._release()

    def __del__(self):
        self.close()


def ms_setup(ctx: Context, indicator, kind: str, moduli, C0, op_tol: float = 1e-10, interleaved: bool = True,
             op_cross: bool = False, op_prec: int = PREC_F64) -> MSOps:
    """Operator trains of an RVE (the setup of ms_homogenize) as a handle that
    ms_homogenize(..., ops=handle) reuses; same arguments as ms_homogenize,
    op_prec PREC_F32 (op_tol >= 1e-7) for the dense TT-SVDs in float."""
    import time as _time
    rve, keep = _rve(indicator, kind, moduli, interleaved, op_cross)
    nc = rve.ncomp
    C0a = np.ascontiguousarray(np.asarray(C0, dtype=np.float64).reshape(nc, nc))
    h = _P()
    t0 = _time.perf_counter()
    _check(_lib.ms_setup(ctx.h, C.byref(rve), C0a.ctypes.data_as(C.POINTER(C.c_double)), float(op_tol),
                         int(op_prec), C.byref(h)), "ms_setup")
    return MSOps(ctx, h, nc, (_time.perf_counter() - t0) * 1e3)


def ms_homogenize(ctx: Context, indicator: np.ndarray, kind: str, moduli, C0, tol: float, max_rank: int,
                  eps: float = 1e-6, op_tol: float = 1e-10, prec: int = PREC_F64, max_iter: int = 100,
                  oversample: int = 8, load_mask: int | None = None, interleaved: bool = True,
                  min_iter: int = 1, seed: int = 12345, predictor: "MLP | None" = None, trace_cap: int = 0,
                  op_cross: bool = False, green_amen: bool = False, return_strain: bool = False,
                  lc_workers: int = 1, warm_iter: int = 0, ops: "MSOps | None" = None):
    """Effective tensor of a two-phase RVE (phase 2 where indicator == 1).

    kind "scalar": moduli = (k1, k2), C0 = 3x3; kind "elastic": moduli =
    (lam1, mu1, lam2, mu2), C0 = Voigt 6x6.  `indicator` is a dense
    (Nx, Ny, Nz) image or a Boxes / Ellipsoids geometry (phase train by TT-cross);
    op_cross builds the Green operator train by TT-cross at any size (it is
    always so above 2^27 voxels); green_amen applies it by AMEn;
    return_strain puts the converged strain train of the last load case in
    report.strain (see contract_voxels); lc_workers solves that many load
    cases at the same time on their own streams (operators built once);
    report.timed_ms times the iterations after the first warm_iter of every
    load case; ops (from ms_setup) reuses operator trains built before, and
    indicator, moduli, C0, op_tol, interleaved and op_cross are then those of
    the setup.  Returns (C_eff, report)."""
    if ops is not None:
        nc = ops.ncomp
        C0a = None
    else:
        rve, keep = _rve(indicator, kind, moduli, interleaved, op_cross)
        nc = rve.ncomp
        C0a = np.ascontiguousarray(np.asarray(C0, dtype=np.float64).reshape(nc, nc))
    o = MSOpts()
    o.prec = int(prec)
    o.eps = float(eps)
    o.op_tol = float(op_tol)
    o.max_iter = int(max_iter)
    o.oversample = int(oversample)
    o.load_mask = int(load_mask if load_mask is not None else (1 << nc) - 1)
    o.min_iter = int(min_iter)
    o.seed = int(seed)
    o.predictor = predictor.h if predictor is not None else None
    trace = np.zeros((max(trace_cap, 1), MLP_FEATURES + 1), dtype=np.float32)
    o.trace = _fptr(trace) if trace_cap > 0 else None
    o.trace_cap = int(trace_cap)
    o.green_amen = 1 if green_amen else 0
    o.lc_workers = int(lc_workers)
    o.warm_iter = int(warm_iter)
    strain = _P()
    o.strain = C.pointer(strain) if return_strain else None
    out = np.zeros((nc, nc), dtype=np.float64)
    rep = MSReport()
    if ops is not None:
        _check(_lib.ms_homogenize_ops(ctx.h, ops.h, float(tol), int(max_rank), C.byref(o),
                                      out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(rep)), "ms_homogenize_ops")
    else:
        _check(_lib.ms_homogenize(ctx.h, C.byref(rve), C0a.ctypes.data_as(C.POINTER(C.c_double)), float(tol),
                                  int(max_rank), C.byref(o), out.ctypes.data_as(C.POINTER(C.c_double)),
                                  C.byref(rep)), "ms_homogenize")
    if trace_cap > 0:
        rep.trace_rows = trace[:rep.trace_len].copy()
    if return_strain:
        rep.strain = TT(ctx, strain) if strain.value else None
    return out, rep
