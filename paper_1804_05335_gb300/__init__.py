"""Python binding of libfdas, the sm_103a FDAS correlation library.

The functions here carry the C ABI's names (include/fdas.h) and only marshal
arguments: torch tensors supply device memory and the current CUDA stream,
and every step of the search runs in the library's kernels.  There is no CPU
fallback: if libfdas.so is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

__all__ = [
    "FdasError", "fdas_params", "fdas_cand", "fdas_fused_threshold", "load_library", "lib_path",
    "params", "fdas_strerror", "fdas_version", "fdas_half_width", "fdas_num_templates",
    "fdas_bank_rows", "fdas_bank_floats", "fdas_num_segments", "fdas_plane_width", "fdas_make_templates",
    "fdas_normalise_workspace_bytes", "fdas_normalise", "fdas_normalise_noalloc",
    "fdas_bluestein_bytes", "fdas_bluestein_prepare", "fdas_normalise_prepared",
    "fdas_correlate", "fdas_correlate_split", "fdas_threshold", "FDAS_NOALLOC_MAX_N",
    "fdas_debug_wait_timeout",
    "fdas_template_groups", "FDAS_MAX_GROUPS",
    "fdas_correlate_plane16", "FDAS_PLANE_F16", "FDAS_PLANE_BF16", "fdas_harmonic_sum",
    "fdas_harmonic_plan_bytes", "fdas_harmonic_plan", "fdas_harmonic_sum_planned", "FDAS_STATUS_BADPLAN",
    "fdas_noise_means",
    "FDAS_PREC_FP32", "FDAS_PREC_FP16_SPLIT", "FDAS_PREC_BF16_SPLIT", "FDAS_PREC_BF16_SPLIT3",
    "fdas_refine_fwd", "fdas_refine_bwd", "fdas_refine", "fdas_trial", "fdas_tuning",
    "fdas_batch_plan", "fdas_correlate_batched",
    "header_functions", "FDAS_CAND_PEAK", "FDAS_STATUS_OVERFLOW", "FDAS_STATUS_TIMEOUT",
    "FDAS_OK", "FDAS_E_INVAL", "FDAS_E_CUDA", "FDAS_E_OVERFLOW", "FDAS_E_TIMEOUT",
    "FDAS_E_UNSUPPORTED",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libfdas.so")
_HEADER = os.path.join(os.path.dirname(_HERE), "include", "fdas.h")

FDAS_OK = 0
FDAS_E_INVAL = -1
FDAS_E_CUDA = -2
FDAS_E_OVERFLOW = -3
FDAS_E_TIMEOUT = -4
FDAS_E_UNSUPPORTED = -5
FDAS_STATUS_TIMEOUT = 1
FDAS_STATUS_OVERFLOW = 2
FDAS_STATUS_BADPLAN = 4
FDAS_CAND_PEAK = 1
FDAS_NOALLOC_MAX_N = 1 << 20
FDAS_MAX_GROUPS = 4
FDAS_PLANE_F16 = 1
FDAS_PLANE_BF16 = 2
FDAS_PREC_FP32 = 0
FDAS_PREC_FP16_SPLIT = 1
FDAS_PREC_BF16_SPLIT = 2
FDAS_PREC_BF16_SPLIT3 = 3

c_i32, c_i64, c_f32, c_vp, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t


class fdas_params(ctypes.Structure):
    _fields_ = [("L", c_i32), ("M", c_i32), ("zmin", c_i32), ("zmax", c_i32),
                ("zstep", c_i32), ("interbin", c_i32)]


class fdas_cand(ctypes.Structure):
    _fields_ = [("z_idx", c_i32), ("col", c_i32), ("power", c_f32), ("flags", c_i32)]


class fdas_fused_threshold(ctypes.Structure):
    _fields_ = [("thr", c_f32), ("out", c_vp), ("cap", c_i32), ("count", c_vp)]


class fdas_trial(ctypes.Structure):
    _fields_ = [("spec", c_vp), ("nb", c_i64), ("plane", c_vp), ("row_stride", c_i64),
                ("item_begin", c_i64)]


class fdas_tuning(ctypes.Structure):
    _fields_ = [("ctas_per_sm", c_i32), ("templates_per_block", c_i32)]


class FdasError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s: %s (%d)" % (what, _strerror(code), code))
        self.code = code


_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libfdas.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libfdas.so is not built (%s); run __graft_entry__.build()" % _LIB_PATH)
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "fdas_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "fdas_version": (ctypes.c_char_p, []),
        "fdas_half_width": (c_i32, [c_i32]),
        "fdas_num_templates": (c_i32, [P(fdas_params)]),
        "fdas_bank_rows": (c_i32, [P(fdas_params)]),
        "fdas_num_segments": (c_i64, [P(fdas_params), c_i64]),
        "fdas_bank_floats": (c_i64, [P(fdas_params)]),
        "fdas_plane_width": (c_i64, [P(fdas_params), c_i64]),
        "fdas_template_groups": (c_i32, [P(fdas_params), c_vp, c_vp, c_vp]),
        "fdas_make_templates": (ctypes.c_int, [P(fdas_params), c_vp, c_vp]),
        "fdas_normalise_workspace_bytes": (c_sz, [c_i64]),
        "fdas_normalise": (ctypes.c_int, [c_vp, c_i64, c_i32, c_vp, c_vp, c_sz, c_vp]),
        "fdas_normalise_noalloc": (ctypes.c_int, [c_vp, c_i64, c_i32, c_vp, c_vp]),
        "fdas_bluestein_bytes": (c_sz, [c_i64]),
        "fdas_bluestein_prepare": (ctypes.c_int, [c_i64, c_vp, c_vp, c_sz, c_vp]),
        "fdas_normalise_prepared": (ctypes.c_int, [c_vp, c_i64, c_i32, c_vp, c_vp, c_sz, c_vp,
                                                   c_vp]),
        "fdas_correlate": (ctypes.c_int, [P(fdas_params), c_vp, c_i64, c_vp, c_vp, c_i64,
                                          P(fdas_fused_threshold), c_vp, c_vp]),
        "fdas_correlate_split": (ctypes.c_int, [P(fdas_params), c_i32, c_vp, c_i64, c_vp, c_vp,
                                                c_i64, P(fdas_fused_threshold), c_vp, c_vp]),
        "fdas_debug_wait_timeout": (ctypes.c_int, [P(fdas_params), c_vp, c_i64, c_vp, c_vp, c_i64,
                                                   ctypes.c_uint32, c_vp, c_vp]),
        "fdas_correlate_plane16": (ctypes.c_int, [P(fdas_params), c_i32, c_vp, c_i64, c_vp, c_vp,
                                                  c_i64, P(fdas_fused_threshold), c_vp, c_vp]),
        "fdas_harmonic_sum": (ctypes.c_int, [P(fdas_params), c_i32, c_vp, c_i64, c_i64, c_i32,
                                             c_vp, c_vp, c_i32, c_vp, c_vp, c_vp]),
        "fdas_harmonic_plan_bytes": (c_sz, [P(fdas_params), c_i64]),
        "fdas_harmonic_plan": (ctypes.c_int, [P(fdas_params), c_i64, c_vp, c_sz]),
        "fdas_harmonic_sum_planned": (ctypes.c_int, [P(fdas_params), c_i32, c_vp, c_i64, c_i64,
                                                     c_i32, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp,
                                                     c_sz, c_vp]),
        "fdas_noise_means": (ctypes.c_int, [P(fdas_params), c_vp, c_vp]),
        "fdas_threshold": (ctypes.c_int, [c_vp, c_i32, c_i64, c_i64, c_f32, c_i32, c_vp, c_i32,
                                          c_vp, c_vp, c_vp]),
        "fdas_batch_plan": (c_i64, [P(fdas_params), P(fdas_trial), c_i32]),
        "fdas_correlate_batched": (ctypes.c_int, [P(fdas_params), c_vp, c_i32, c_i64, c_vp,
                                                  P(fdas_fused_threshold), P(fdas_tuning), c_vp,
                                                  c_vp]),
        "fdas_refine_fwd": (ctypes.c_int, [c_vp, c_i64, c_vp, c_vp, c_i32, c_i32, c_vp, c_vp,
                                           c_vp, c_vp, c_vp]),
        "fdas_refine_bwd": (ctypes.c_int, [c_vp, c_i64, c_vp, c_vp, c_i32, c_i32, c_vp, c_vp,
                                           c_vp, c_vp]),
        "fdas_refine": (ctypes.c_int, [c_vp, c_i64, c_vp, c_vp, c_i32, c_i32, c_i32,
                                       ctypes.c_double, ctypes.c_double, c_vp, c_vp, c_vp, c_vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_functions():
    """Names of the functions declared in include/fdas.h."""
    txt = open(_HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fdas_[a-z0-9_]+)\s*\(", txt)))


def _strerror(code: int) -> str:
    try:
        return load_library().fdas_strerror(int(code)).decode()
    except Exception:  # noqa: BLE001 - only used while formatting an error
        return "error"


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise FdasError(int(rc), what)
    return rc


def _ptr(t) -> int:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return int(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def params(L=2048, M=256, zmin=-200, zmax=200, zstep=2, interbin=1) -> fdas_params:
    return fdas_params(int(L), int(M), int(zmin), int(zmax), int(zstep), int(interbin))


def fdas_strerror(code: int) -> str:
    return load_library().fdas_strerror(int(code)).decode()


def fdas_version() -> str:
    return load_library().fdas_version().decode()


def fdas_half_width(z: int) -> int:
    return int(load_library().fdas_half_width(int(z)))


def fdas_num_templates(p: fdas_params) -> int:
    return _check(load_library().fdas_num_templates(ctypes.byref(p)), "fdas_num_templates")


def fdas_bank_rows(p: fdas_params) -> int:
    return _check(load_library().fdas_bank_rows(ctypes.byref(p)), "fdas_bank_rows")


def fdas_bank_floats(p: fdas_params) -> int:
    return _check(load_library().fdas_bank_floats(ctypes.byref(p)), "fdas_bank_floats")


def fdas_num_segments(p: fdas_params, nb: int) -> int:
    return _check(load_library().fdas_num_segments(ctypes.byref(p), int(nb)), "fdas_num_segments")


def fdas_plane_width(p: fdas_params, nb: int) -> int:
    return _check(load_library().fdas_plane_width(ctypes.byref(p), int(nb)), "fdas_plane_width")


def fdas_template_groups(p: fdas_params):
    """[(overlap, first bank row, plane rows), ...] of the convolver's template groups."""
    ov = (c_i32 * FDAS_MAX_GROUPS)()
    fr = (c_i32 * FDAS_MAX_GROUPS)()
    ct = (c_i32 * FDAS_MAX_GROUPS)()
    n = _check(load_library().fdas_template_groups(ctypes.byref(p), ov, fr, ct),
               "fdas_template_groups")
    return [(ov[k], fr[k], ct[k]) for k in range(n)]


def fdas_make_templates(p: fdas_params, bank, stream=None) -> None:
    """bank: device float32 tensor of fdas_bank_floats(p) elements."""
    _check(load_library().fdas_make_templates(ctypes.byref(p), _ptr(bank), _stream(stream)),
           "fdas_make_templates")


def fdas_normalise_workspace_bytes(n: int) -> int:
    return int(load_library().fdas_normalise_workspace_bytes(int(n)))


def fdas_normalise(series, n: int, median_block: int, spec, work, work_bytes: int,
                   stream=None) -> None:
    """series: device float32[n]; spec: device complex64[n/2] (or float32[n])."""
    _check(load_library().fdas_normalise(_ptr(series), int(n), int(median_block), _ptr(spec),
                                         _ptr(work), int(work_bytes), _stream(stream)),
           "fdas_normalise")


def fdas_bluestein_bytes(n: int) -> int:
    return int(load_library().fdas_bluestein_bytes(int(n)))


def fdas_bluestein_prepare(n: int, chirp_spec, work, work_bytes: int, stream=None) -> None:
    """chirp_spec: device buffer of fdas_bluestein_bytes(n) bytes (written)."""
    _check(load_library().fdas_bluestein_prepare(int(n), _ptr(chirp_spec), _ptr(work),
                                                 int(work_bytes), _stream(stream)),
           "fdas_bluestein_prepare")


def fdas_normalise_prepared(series, n: int, median_block: int, spec, work, work_bytes: int,
                            chirp_spec, stream=None) -> None:
    """fdas_normalise with the Bluestein kernel spectrum from fdas_bluestein_prepare."""
    _check(load_library().fdas_normalise_prepared(_ptr(series), int(n), int(median_block),
                                                  _ptr(spec), _ptr(work), int(work_bytes),
                                                  _ptr(chirp_spec), _stream(stream)),
           "fdas_normalise_prepared")


def fdas_normalise_noalloc(series, n: int, median_block: int, spec, stream=None) -> None:
    """fdas_normalise with the library's fixed device workspace (n <= 2^20).

    For callers that must not allocate device memory at call time; see the
    declaration in include/fdas.h for the limits (one shared workspace per
    GPU: calls that can overlap on the GPU race).
    """
    _check(load_library().fdas_normalise_noalloc(_ptr(series), int(n), int(median_block),
                                                 _ptr(spec), _stream(stream)),
           "fdas_normalise_noalloc")


def fdas_correlate(p: fdas_params, spec, nb: int, bank, plane, row_stride: int,
                   fused: fdas_fused_threshold | None = None, status=None, stream=None) -> None:
    f = ctypes.byref(fused) if fused is not None else None
    _check(load_library().fdas_correlate(ctypes.byref(p), _ptr(spec), int(nb), _ptr(bank),
                                         _ptr(plane), int(row_stride), f, _ptr(status),
                                         _stream(stream)), "fdas_correlate")


def fdas_correlate_plane16(p: fdas_params, ptype: int, spec, nb: int, bank, plane, row_stride: int,
                           fused: fdas_fused_threshold | None = None, status=None,
                           stream=None) -> None:
    f = ctypes.byref(fused) if fused is not None else None
    _check(load_library().fdas_correlate_plane16(ctypes.byref(p), int(ptype), _ptr(spec),
                                                 int(nb), _ptr(bank), _ptr(plane),
                                                 int(row_stride), f, _ptr(status),
                                                 _stream(stream)), "fdas_correlate_plane16")


def fdas_harmonic_sum(p: fdas_params, plane_type: int, plane, width: int, row_stride: int,
                      thresholds, out, cap: int, count, status=None, stream=None) -> None:
    """Harmonic sums H = 2, 4, 8 (one threshold per level) with candidates in out."""
    thr = (c_f32 * 3)(*[float(v) for v in thresholds])
    _check(load_library().fdas_harmonic_sum(ctypes.byref(p), int(plane_type), _ptr(plane),
                                            int(width), int(row_stride), len(thresholds), thr,
                                            _ptr(out), int(cap), _ptr(count), _ptr(status),
                                            _stream(stream)), "fdas_harmonic_sum")


def fdas_harmonic_plan_bytes(p: fdas_params, width: int) -> int:
    """Device bytes of the ray-order plan for grid p and plane width (0: invalid)."""
    return int(load_library().fdas_harmonic_plan_bytes(ctypes.byref(p), int(width)))


def fdas_harmonic_plan(p: fdas_params, width: int, plan, plan_bytes: int) -> None:
    """Build the ray-order plan into device memory `plan` (returns when copied)."""
    _check(load_library().fdas_harmonic_plan(ctypes.byref(p), int(width), _ptr(plan),
                                             int(plan_bytes)), "fdas_harmonic_plan")


def fdas_harmonic_sum_planned(p: fdas_params, plane_type: int, plane, width: int,
                              row_stride: int, thresholds, out, cap: int, count, plan,
                              plan_bytes: int, status=None, stream=None) -> None:
    """fdas_harmonic_sum with its blocks taken in the plan's ray order."""
    thr = (c_f32 * 3)(*[float(v) for v in thresholds])
    _check(load_library().fdas_harmonic_sum_planned(
        ctypes.byref(p), int(plane_type), _ptr(plane), int(width), int(row_stride),
        len(thresholds), thr, _ptr(out), int(cap), _ptr(count), _ptr(status), _ptr(plan),
        int(plan_bytes), _stream(stream)), "fdas_harmonic_sum_planned")


def fdas_noise_means(p: fdas_params, means, stream=None) -> None:
    _check(load_library().fdas_noise_means(ctypes.byref(p), _ptr(means), _stream(stream)),
           "fdas_noise_means")


def fdas_correlate_split(p: fdas_params, prec: int, spec, nb: int, bank, plane, row_stride: int,
                         fused: fdas_fused_threshold | None = None, status=None,
                         stream=None) -> None:
    f = ctypes.byref(fused) if fused is not None else None
    _check(load_library().fdas_correlate_split(ctypes.byref(p), int(prec), _ptr(spec), int(nb),
                                               _ptr(bank), _ptr(plane), int(row_stride), f,
                                               _ptr(status), _stream(stream)),
           "fdas_correlate_split")


def fdas_debug_wait_timeout(p: fdas_params, spec, nb: int, bank, plane, row_stride: int,
                            polls: int, status, stream=None) -> None:
    _check(load_library().fdas_debug_wait_timeout(ctypes.byref(p), _ptr(spec), int(nb), _ptr(bank),
                                                  _ptr(plane), int(row_stride), int(polls),
                                                  _ptr(status), _stream(stream)),
           "fdas_debug_wait_timeout")


def fdas_threshold(plane, rows: int, width: int, row_stride: int, thr: float, want_flags: int,
                   out, cap: int, count, status=None, stream=None) -> None:
    _check(load_library().fdas_threshold(_ptr(plane), int(rows), int(width), int(row_stride),
                                         float(thr), int(want_flags), _ptr(out), int(cap),
                                         _ptr(count), _ptr(status), _stream(stream)),
           "fdas_threshold")


def fdas_refine_fwd(spec, nb: int, r, z, ncand: int, m: int, P, dPdr=None, dPdz=None, S=None,
                    stream=None) -> None:
    _check(load_library().fdas_refine_fwd(_ptr(spec), int(nb), _ptr(r), _ptr(z), int(ncand),
                                          int(m), _ptr(P), _ptr(dPdr), _ptr(dPdz), _ptr(S),
                                          _stream(stream)), "fdas_refine_fwd")


def fdas_refine_bwd(spec, nb: int, r, z, ncand: int, m: int, S, gP, grad_spec,
                    stream=None) -> None:
    _check(load_library().fdas_refine_bwd(_ptr(spec), int(nb), _ptr(r), _ptr(z), int(ncand),
                                          int(m), _ptr(S), _ptr(gP), _ptr(grad_spec),
                                          _stream(stream)), "fdas_refine_bwd")


def fdas_refine(spec, nb: int, r_in, z_in, ncand: int, m: int, steps: int, lr_r: float,
                lr_z: float, r_out, z_out, P_out, stream=None) -> None:
    _check(load_library().fdas_refine(_ptr(spec), int(nb), _ptr(r_in), _ptr(z_in), int(ncand),
                                      int(m), int(steps), float(lr_r), float(lr_z), _ptr(r_out),
                                      _ptr(z_out), _ptr(P_out), _stream(stream)), "fdas_refine")


def fdas_batch_plan(p: fdas_params, trials) -> int:
    """trials: ctypes array of fdas_trial (host); fills item_begin, returns total items."""
    return _check(load_library().fdas_batch_plan(ctypes.byref(p), trials, len(trials)),
                  "fdas_batch_plan")


def fdas_correlate_batched(p: fdas_params, trials_dev, ntrials: int, total_items: int, bank,
                           fused: fdas_fused_threshold | None = None, ctas_per_sm: int = 0,
                           status=None, stream=None, templates_per_block: int = 0) -> None:
    f = ctypes.byref(fused) if fused is not None else None
    tun = fdas_tuning(int(ctas_per_sm), int(templates_per_block))
    _check(load_library().fdas_correlate_batched(ctypes.byref(p), _ptr(trials_dev), int(ntrials),
                                                 int(total_items), _ptr(bank), f,
                                                 ctypes.byref(tun), _ptr(status),
                                                 _stream(stream)), "fdas_correlate_batched")
