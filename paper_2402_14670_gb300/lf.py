"""Python binding of the C ABI in include/lf.h (argument marshalling only).

The functions keep the C names (lf_create, lf_pack_hits, lf_find_tracks,
lf_find_tracks_batched, lf_debug_stages, lf_sync_status, lf_destroy); every
step of the path runs in the CUDA library.  ``Tracker`` wraps them for torch
tensors: it allocates outputs with torch and passes raw device pointers and
the current CUDA stream.

Importing this module loads ``liblf.so``; it raises if the library has not
been built (there is no fallback of any kind).
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblf.so")
NL = 12
NB = 24

LF_OK, LF_ERR_ARG, LF_ERR_CUDA, LF_ERR_OOM, LF_ERR_CAPACITY, LF_ERR_TIMEOUT, LF_ERR_INTERNAL = range(7)
_STATUS = {0: "LF_OK", 1: "LF_ERR_ARG", 2: "LF_ERR_CUDA", 3: "LF_ERR_OOM", 4: "LF_ERR_CAPACITY",
           5: "LF_ERR_TIMEOUT", 6: "LF_ERR_INTERNAL"}

if not os.path.exists(LIB_PATH):
    raise ImportError("liblf.so is not built: run paper_2402_14670_gb300.build.build() "
                      "(the CUDA library is required; there is no CPU path)")
_lib = C.CDLL(LIB_PATH)

_P = C.c_void_p


class lf_geometry(C.Structure):
    _fields_ = [("z", C.c_float * NL), ("dxdy", C.c_float * NL), ("z_state", C.c_float),
                ("z_magnet", C.c_float), ("z_ref", C.c_float), ("kappa", C.c_float), ("gamma", C.c_float),
                ("dratio", C.c_float), ("polarity", C.c_int32)]


class lf_params(C.Structure):
    _fields_ = [("xtol_c", C.c_float), ("xtol_p", C.c_float), ("x_asym", C.c_float), ("uv_tol", C.c_float),
                ("n_hits_window", C.c_int32), ("n_triplets", C.c_int32), ("min_hits", C.c_int32),
                ("K_first", C.c_float), ("K_last", C.c_float), ("p_bend", C.c_float),
                ("magtol_min", C.c_float), ("magtol_max", C.c_float), ("magtol_c", C.c_float),
                ("magtol_tx", C.c_float), ("T_triplet", C.c_float), ("T_x", C.c_float),
                ("T_uv_scale", C.c_float), ("T_uv_min", C.c_float), ("T_ty", C.c_float), ("T_y", C.c_float),
                ("T_Q", C.c_float), ("C_n", C.c_float * 4), ("no_ut", C.c_int32), ("p_min", C.c_float),
                ("pt_min", C.c_float), ("x_overlap", C.c_float), ("tol_c", C.c_float * 8),
                ("qop_poly", C.c_int32), ("qop_c", (C.c_float * 10) * 5)]


class lf_raw_hits(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("n_hits", C.c_int32), ("raw_offsets", _P), ("x", _P), ("z", _P),
                ("dxdy", _P), ("w", _P), ("plane", _P)]


class lf_packed(C.Structure):
    _fields_ = [("hit_offsets", _P), ("x", _P), ("z", _P), ("dxdy", _P), ("w", _P), ("layer", _P), ("perm", _P),
                ("x_coarse", _P)]


class lf_batch(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("n_hits", C.c_int32), ("n_tracks", C.c_int32), ("hit_offsets", _P),
                ("x", _P), ("z", _P), ("dxdy", _P), ("w", _P), ("trk_offsets", _P), ("sx", _P), ("sy", _P),
                ("stx", _P), ("sty", _P), ("sqop", _P), ("x_coarse", _P)]


class lf_output(C.Structure):
    _fields_ = [("found", _P), ("nhits", _P), ("hit_idx", _P), ("state", _P), ("quality", _P),
                ("out_offsets", _P), ("out_trk", _P), ("n_out", _P)]


class lf_gather(C.Structure):
    _fields_ = [("hit_src", _P), ("trk_src", _P), ("sx", _P), ("sy", _P), ("stx", _P), ("sty", _P), ("sqop", _P)]


class lf_host_batch(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("n_hits", C.c_int32), ("n_tracks", C.c_int32), ("raw_offsets", _P),
                ("x", _P), ("z", _P), ("dxdy", _P), ("w", _P), ("plane", _P), ("trk_offsets", _P), ("sx", _P),
                ("sy", _P), ("stx", _P), ("sty", _P), ("sqop", _P)]


class lf_host_output(C.Structure):
    _fields_ = [("found", _P), ("nhits", _P), ("hit_idx", _P), ("state", _P), ("quality", _P)]


class lf_tuning(C.Structure):
    _fields_ = [("warps_per_block", C.c_int32), ("blocks_per_sm", C.c_int32), ("grain", C.c_int32),
                ("queue", C.c_int32), ("windows_bps", C.c_int32), ("triplets_bps", C.c_int32),
                ("extend_bps", C.c_int32), ("triplet_prefilter", C.c_int32),
                ("extend_form", C.c_int32)]


def coarse_count(n_hits: int) -> int:
    """Length of the coarse index of n_hits packed hits (every 32nd x)."""
    return (int(n_hits) + 31) // 32 + 1


def tuning_struct(tuning: Optional[dict]) -> Optional[lf_tuning]:
    """lf_tuning from a dict of its fields (missing fields 0 = defaults)."""
    if not tuning:
        return None
    return lf_tuning(*(int(tuning.get(f, 0)) for f, _ in lf_tuning._fields_))


_lib.lf_create.argtypes = [C.POINTER(lf_geometry), C.POINTER(lf_params), C.POINTER(_P)]
_lib.lf_create.restype = C.c_int
_lib.lf_destroy.argtypes = [_P]
_lib.lf_destroy.restype = None
_lib.lf_last_error.argtypes = [_P]
_lib.lf_last_error.restype = C.c_char_p
_lib.lf_device_sm_count.argtypes = []
_lib.lf_device_sm_count.restype = C.c_int32
_lib.lf_device_host_numa.argtypes = []
_lib.lf_device_host_numa.restype = C.c_int32
_lib.lf_pack_hits.argtypes = [_P, C.POINTER(lf_raw_hits), C.POINTER(lf_packed), _P]
_lib.lf_pack_hits.restype = C.c_int
_lib.lf_find_tracks.argtypes = [_P, C.POINTER(lf_batch), C.POINTER(lf_output), _P]
_lib.lf_find_tracks.restype = C.c_int
_lib.lf_find_tracks_batched.argtypes = [_P, C.POINTER(lf_batch), C.POINTER(lf_output), C.POINTER(lf_tuning), _P]
_lib.lf_find_tracks_batched.restype = C.c_int
_lib.lf_debug_stages.argtypes = [_P, C.POINTER(lf_batch), _P, _P, _P, _P, _P, _P]
_lib.lf_debug_stages.restype = C.c_int
_lib.lf_validate_batch.argtypes = [_P, C.POINTER(lf_batch), _P]
_lib.lf_validate_batch.restype = C.c_int
_lib.lf_debug_triplets.argtypes = [_P, C.POINTER(lf_batch), _P, _P, _P, _P, _P]
_lib.lf_debug_triplets.restype = C.c_int
_lib.lf_sync_status.argtypes = [_P, _P, C.POINTER(C.c_int32)]
_lib.lf_sync_status.restype = C.c_int
_lib.lf_process_host.argtypes = [_P, C.POINTER(lf_host_batch), C.POINTER(lf_host_output), C.POINTER(lf_tuning),
                                 C.c_int64]
_lib.lf_process_host.restype = C.c_int

_lib.lf_process_slot.argtypes = [_P, C.POINTER(lf_raw_hits), C.POINTER(lf_packed), C.POINTER(lf_batch),
                                 C.POINTER(lf_gather), _P, C.POINTER(lf_output), C.POINTER(lf_tuning), _P]
_lib.lf_process_slot.restype = C.c_int
_lib.lf_graph_count.argtypes = [_P]
_lib.lf_graph_count.restype = C.c_int64
_lib.lf_find_tracks_static.argtypes = [C.POINTER(lf_geometry), C.POINTER(lf_params), C.POINTER(lf_batch),
                                       C.POINTER(lf_output), _P]
_lib.lf_find_tracks_static.restype = C.c_int
_lib.lf_reserve.argtypes = [_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(lf_tuning)]
_lib.lf_reserve.restype = C.c_int
_lib.lf_host_alloc.argtypes = [C.c_size_t, C.POINTER(_P)]
_lib.lf_host_alloc.restype = C.c_int
_lib.lf_host_free.argtypes = [_P]
_lib.lf_host_free.restype = None

EXPORTED = ["lf_create", "lf_destroy", "lf_last_error", "lf_device_sm_count", "lf_pack_hits", "lf_find_tracks",
            "lf_find_tracks_batched", "lf_debug_stages", "lf_debug_triplets", "lf_validate_batch", "lf_sync_status",
            "lf_process_host",
            "lf_find_tracks_static", "lf_host_alloc", "lf_host_free", "lf_reserve", "lf_device_host_numa",
            "lf_process_slot", "lf_graph_count"]


class LFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


# ------------------------------------------------------------- defaults

def default_geometry() -> dict:
    """Synthetic detector: three x-u-v-x stations, stereo +-tan(5 deg),
    kick plane at 5200 mm, reference plane at 8520 mm (Sec. "Extending
    triplets to other layers")."""
    t = float(np.float32(math.tan(math.radians(5.0))))
    kinds = ("x", "u", "v", "x") * 3
    return dict(z=[7826.0, 7896.0, 7966.0, 8036.0, 8508.0, 8578.0, 8648.0, 8718.0,
                   9193.0, 9263.0, 9333.0, 9403.0],
                dxdy=[0.0 if k == "x" else (t if k == "u" else -t) for k in kinds],
                z_state=2700.0, z_magnet=5200.0, z_ref=8520.0, kappa=1.2, gamma=2.4e-9, dratio=4e-4,
                polarity=1)


def default_params(paper_K: bool = False) -> dict:
    """'Forward' column of Table tolerances and Table C_nhits.  K_x1 = 1
    unless paper_K (the synthetic detector has no field in the T stations);
    the magnet tolerance clamp(8 + 96/p + 10|t_x|, 8, 40) mm and
    T_uv = max(2, 50 (|t_x| + |t_y|)) are the readings of what the paper
    leaves open."""
    return dict(xtol_c=150.0, xtol_p=2000.0, x_asym=100.0, uv_tol=800.0, n_hits_window=32, n_triplets=12,
                min_hits=9, K_first=1.00177513 if paper_K else 1.0, K_last=1.00142634 if paper_K else 1.0,
                p_bend=5.0, magtol_min=8.0, magtol_max=40.0, magtol_c=96.0, magtol_tx=10.0, T_triplet=8.0,
                T_x=2.0, T_uv_scale=50.0, T_uv_min=2.0, T_ty=0.02, T_y=800.0, T_Q=0.5,
                C_n=[5.0, 1.0, 0.8, 0.5], no_ut=0, p_min=5.0, pt_min=1.0, x_overlap=5.0,
                tol_c=[4824.3, 426.3, 7071.1, 12080.4, 14077.8, 13909.3, 9315.3, 3209.5],
                qop_poly=0, qop_c=[[0.0] * 10 for _ in range(5)])


def qop_poly_params(coefficients, base: Optional[dict] = None) -> dict:
    """Parameters with q/p from Eq. pt_kick and the polynomial field integral
    (Sec. "Calculation of momentum and track states"); coefficients[5][10]
    as fitted by qop_fit.fit_qop_poly."""
    p = dict(base or default_params())
    p.update(qop_poly=1, qop_c=[[float(v) for v in row] for row in np.asarray(coefficients, np.float32)])
    return p


def no_ut_params() -> dict:
    """The no-UT variant (Sec. "No-UT tuning"): VELO tracks without a
    momentum, windows from Eq. tol_noUT (Table poly_tol) at the tighter of
    p = 5 GeV and pT = 1 GeV, two one-sided windows overlapping by 5 mm, u/v
    tolerance 1200 mm, a fixed 10 mm magnet tolerance, and the "Forward
    no-UT" column of Table tolerances (T_uv = max(T_x, 15 (|t_x| + |t_y|)))."""
    p = default_params()
    p.update(no_ut=1, uv_tol=1200.0, n_hits_window=64, n_triplets=20, magtol_min=10.0, magtol_max=10.0,
             magtol_c=0.0, magtol_tx=0.0, T_triplet=2.0, T_x=0.5, T_uv_scale=15.0, T_uv_min=0.5, T_ty=0.003,
             T_y=800.0, T_Q=0.5)
    return p


def _geometry(g: dict) -> lf_geometry:
    s = lf_geometry()
    s.z[:] = [float(v) for v in g["z"]]
    s.dxdy[:] = [float(v) for v in g["dxdy"]]
    for k in ("z_state", "z_magnet", "z_ref", "kappa", "gamma", "dratio"):
        setattr(s, k, float(g[k]))
    s.polarity = int(g["polarity"])
    return s


def _params(p: dict) -> lf_params:
    s = lf_params()
    for name, _ in lf_params._fields_:
        if name in ("C_n", "tol_c"):
            getattr(s, name)[:] = [float(v) for v in p[name]]
        elif name == "qop_c":
            c = p.get("qop_c", [[0.0] * 10 for _ in range(5)])
            for i in range(5):
                s.qop_c[i][:] = [float(v) for v in c[i]]
        elif name == "qop_poly":
            s.qop_poly = int(p.get("qop_poly", 0))
        else:
            setattr(s, name, p[name])
    return s


# ------------------------------------------------------------- C names

def _check(ctx, st):
    if st != LF_OK:
        msg = _lib.lf_last_error(ctx).decode() if ctx else ""
        raise LFError(st, msg)


def lf_create(geometry: Optional[dict] = None, params: Optional[dict] = None):
    g = _geometry(geometry or default_geometry())
    p = _params(params or default_params())
    h = _P()
    st = _lib.lf_create(C.byref(g), C.byref(p), C.byref(h))
    if st != LF_OK:
        raise LFError(st, "lf_create rejected the geometry or parameters")
    return h


def lf_destroy(ctx) -> None:
    _lib.lf_destroy(ctx)


def lf_last_error(ctx) -> str:
    return _lib.lf_last_error(ctx).decode()


def lf_device_sm_count() -> int:
    return int(_lib.lf_device_sm_count())


def lf_device_host_numa() -> int:
    return int(_lib.lf_device_host_numa())


def lf_reserve(ctx, n_events: int, n_hits: int, n_tracks: int, tuning: Optional["lf_tuning"] = None) -> None:
    _check(ctx, _lib.lf_reserve(ctx, int(n_events), int(n_hits), int(n_tracks),
                                C.byref(tuning) if tuning else None))


def lf_host_alloc(nbytes: int) -> int:
    """Page-locked host memory of exactly nbytes (0 when nbytes is 0)."""
    p = _P()
    st = _lib.lf_host_alloc(C.c_size_t(int(nbytes)), C.byref(p))
    if st != LF_OK:
        raise LFError(st, "lf_host_alloc of %d bytes failed" % nbytes)
    return int(p.value or 0)


def lf_host_free(ptr: int) -> None:
    _lib.lf_host_free(_P(ptr) if ptr else None)


class HostArena:
    """Page-locked host memory of an exact size from lf_host_alloc, carved
    into torch tensors (torch's own pinned allocator rounds multi-GB requests
    up to a power of two).  The tensors are views of the arena's memory, not
    owners of it: none may be used after close() (or the end of a ``with``
    block), and no copy from or to them may still be in flight then."""

    def __init__(self, nbytes: int):
        self.nbytes = max(int(nbytes), 4096)
        self.ptr = lf_host_alloc(self.nbytes)
        self.base = torch.frombuffer((C.c_uint8 * self.nbytes).from_address(self.ptr), dtype=torch.uint8)
        self.off = 0

    def take(self, n: int, dtype) -> torch.Tensor:
        esz = torch.empty(0, dtype=dtype).element_size()
        self.off = (self.off + 255) & ~255
        if self.off + n * esz > self.nbytes:
            raise ValueError("host arena exhausted")
        t = self.base[self.off:self.off + n * esz].view(dtype)
        self.off += n * esz
        return t

    def close(self):
        if self.ptr:
            self.base = None
            lf_host_free(self.ptr)
            self.ptr = 0

    def __enter__(self) -> "HostArena":
        return self

    def __exit__(self, *exc) -> None:
        self.close()


def lf_pack_hits(ctx, raw: lf_raw_hits, packed: lf_packed, stream) -> None:
    _check(ctx, _lib.lf_pack_hits(ctx, C.byref(raw), C.byref(packed), stream))


def lf_find_tracks(ctx, batch: lf_batch, out: lf_output, stream) -> None:
    _check(ctx, _lib.lf_find_tracks(ctx, C.byref(batch), C.byref(out), stream))


def lf_find_tracks_batched(ctx, batch: lf_batch, out: lf_output, tuning: Optional[lf_tuning], stream) -> None:
    tp = C.byref(tuning) if tuning is not None else None
    _check(ctx, _lib.lf_find_tracks_batched(ctx, C.byref(batch), C.byref(out), tp, stream))


def lf_process_slot(ctx, raw: lf_raw_hits, packed: lf_packed, batch: lf_batch, gather: Optional[lf_gather],
                    n_events_dev: int, out: lf_output, tuning: Optional[lf_tuning], stream) -> None:
    gp = C.byref(gather) if gather is not None else None
    tp = C.byref(tuning) if tuning is not None else None
    _check(ctx, _lib.lf_process_slot(ctx, C.byref(raw), C.byref(packed), C.byref(batch), gp, _P(n_events_dev),
                                     C.byref(out), tp, stream))


def lf_graph_count(ctx) -> int:
    return int(_lib.lf_graph_count(ctx))


def lf_debug_stages(ctx, batch: lf_batch, win_begin, win_count, n_trip, trip, trip_chi2, stream) -> None:
    _check(ctx, _lib.lf_debug_stages(ctx, C.byref(batch), win_begin, win_count, n_trip, trip, trip_chi2, stream))


def lf_validate_batch(ctx, batch: lf_batch, stream) -> None:
    _check(ctx, _lib.lf_validate_batch(ctx, C.byref(batch), stream))


def lf_debug_triplets(ctx, batch: lf_batch, win_count, n_trip, trip, trip_chi2, stream) -> None:
    _check(ctx, _lib.lf_debug_triplets(ctx, C.byref(batch), win_count, n_trip, trip, trip_chi2, stream))


def lf_process_host(ctx, batch: lf_host_batch, out: lf_host_output, tuning: Optional[lf_tuning],
                    chunk_hits: int = 0) -> None:
    tp = C.byref(tuning) if tuning is not None else None
    _check(ctx, _lib.lf_process_host(ctx, C.byref(batch), C.byref(out), tp, C.c_int64(chunk_hits)))


def lf_find_tracks_static(geometry: dict, params: dict, batch: lf_batch, out: lf_output, stream) -> None:
    """Context-free persistent form for callers that cannot allocate device
    memory (scratch is a fixed static device array; see include/lf.h)."""
    g, p = _geometry(geometry), _params(params)
    st = _lib.lf_find_tracks_static(C.byref(g), C.byref(p), C.byref(batch), C.byref(out), stream)
    if st != LF_OK:
        raise LFError(st, "lf_find_tracks_static")


def lf_sync_status(ctx, stream) -> int:
    f = C.c_int32(0)
    _check(ctx, _lib.lf_sync_status(ctx, stream, C.byref(f)))
    return int(f.value)


# ------------------------------------------------------------- torch layer

def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return _P(t.data_ptr()) if t.numel() else _P(t.data_ptr() or 0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _P(s.cuda_stream)


class Tracker:
    """A library context plus torch-allocated inputs and outputs."""

    def __init__(self, geometry: Optional[dict] = None, params: Optional[dict] = None):
        self.geometry = dict(geometry or default_geometry())
        self.params = dict(params or default_params())
        self.ctx = lf_create(self.geometry, self.params)

    def close(self):
        if self.ctx:
            lf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # raw -> packed
    def pack(self, raw, stream=None, out: Optional[dict] = None) -> dict:
        n_ev, n_h = int(raw.n_events), int(raw.x.numel())
        dev = raw.x.device
        if out is None:
            out = dict(hit_offsets=torch.empty(NB * n_ev + 1, dtype=torch.int32, device=dev),
                       x=torch.empty(n_h, dtype=torch.float32, device=dev),
                       z=torch.empty(n_h, dtype=torch.float32, device=dev),
                       dxdy=torch.empty(n_h, dtype=torch.float32, device=dev),
                       w=torch.empty(n_h, dtype=torch.float32, device=dev),
                       layer=torch.empty(n_h, dtype=torch.uint8, device=dev),
                       perm=torch.empty(n_h, dtype=torch.int32, device=dev),
                       x_coarse=torch.empty(coarse_count(n_h), dtype=torch.float32, device=dev))
        r = lf_raw_hits(n_ev, n_h, _ptr(raw.raw_offsets), _ptr(raw.x), _ptr(raw.z), _ptr(raw.dxdy), _ptr(raw.w),
                        _ptr(raw.plane))
        p = lf_packed(_ptr(out["hit_offsets"]), _ptr(out["x"]), _ptr(out["z"]), _ptr(out["dxdy"]), _ptr(out["w"]),
                      _ptr(out["layer"]), _ptr(out["perm"]), _ptr(out.get("x_coarse")))
        lf_pack_hits(self.ctx, r, p, _stream(stream))
        return out

    @staticmethod
    def batch_struct(packed: dict, states, n_events: int) -> lf_batch:
        return lf_batch(int(n_events), int(packed["x"].numel()), int(states.sx.numel()), _ptr(packed["hit_offsets"]),
                        _ptr(packed["x"]), _ptr(packed["z"]), _ptr(packed["dxdy"]), _ptr(packed["w"]),
                        _ptr(states.trk_offsets), _ptr(states.sx), _ptr(states.sy), _ptr(states.stx),
                        _ptr(states.sty), _ptr(states.sqop), _ptr(packed.get("x_coarse")))

    @staticmethod
    def alloc_output(n_tracks: int, n_events: int, device) -> dict:
        return dict(found=torch.empty(n_tracks, dtype=torch.uint8, device=device),
                    nhits=torch.empty(n_tracks, dtype=torch.uint8, device=device),
                    hit_idx=torch.empty((n_tracks, NL), dtype=torch.int32, device=device),
                    state=torch.empty((n_tracks, 6), dtype=torch.float32, device=device),
                    quality=torch.empty(n_tracks, dtype=torch.float32, device=device),
                    out_offsets=torch.empty(n_events + 1, dtype=torch.int32, device=device),
                    out_trk=torch.empty(max(n_tracks, 1), dtype=torch.int32, device=device),
                    n_out=torch.empty(1, dtype=torch.int32, device=device))

    @staticmethod
    def output_struct(o: dict) -> lf_output:
        return lf_output(_ptr(o["found"]), _ptr(o["nhits"]), _ptr(o["hit_idx"]), _ptr(o["state"]),
                         _ptr(o["quality"]), _ptr(o["out_offsets"]), _ptr(o["out_trk"]), _ptr(o["n_out"]))

    def find(self, packed: dict, states, n_events: int, mode: str = "batched", tuning: Optional[dict] = None,
             stream=None, out: Optional[dict] = None) -> dict:
        b = self.batch_struct(packed, states, n_events)
        if out is None:
            out = self.alloc_output(int(states.sx.numel()), int(n_events), packed["x"].device)
        o = self.output_struct(out)
        if mode == "plain":
            lf_find_tracks(self.ctx, b, o, _stream(stream))
        elif mode == "batched":
            tu = tuning_struct(tuning)
            lf_find_tracks_batched(self.ctx, b, o, tu, _stream(stream))
        else:
            raise ValueError(mode)
        return out

    def debug_stages(self, packed: dict, states, n_events: int, stream=None) -> dict:
        n_t = int(states.sx.numel())
        nt = max(int(self.params["n_triplets"]), 1)
        dev = packed["x"].device
        ns = 2 if self.params.get("no_ut", 0) else 1   # window sets per track, side-major
        d = dict(win_begin=torch.empty((n_t, ns * NL), dtype=torch.int32, device=dev),
                 win_count=torch.empty((n_t, ns * NL), dtype=torch.int32, device=dev),
                 n_trip=torch.empty(n_t, dtype=torch.int32, device=dev),
                 trip=torch.full((n_t, nt, 4), -1, dtype=torch.int32, device=dev),
                 trip_chi2=torch.zeros((n_t, nt), dtype=torch.float32, device=dev))
        b = self.batch_struct(packed, states, n_events)
        lf_debug_stages(self.ctx, b, _ptr(d["win_begin"]), _ptr(d["win_count"]), _ptr(d["n_trip"]),
                        _ptr(d["trip"]), _ptr(d["trip_chi2"]), _stream(stream))
        return d

    def last_triplets(self, packed: dict, states, n_events: int, stream=None) -> dict:
        """Triplet lists the last batched call (stage pipeline) left in the
        context's scratch, decoded without running any stage again."""
        n_t = int(states.sx.numel())
        nt = max(int(self.params["n_triplets"]), 1)
        dev = packed["x"].device
        ns = 2 if self.params.get("no_ut", 0) else 1
        d = dict(win_count=torch.empty((n_t, ns * NL), dtype=torch.int32, device=dev),
                 n_trip=torch.empty(n_t, dtype=torch.int32, device=dev),
                 trip=torch.full((n_t, nt, 4), -1, dtype=torch.int32, device=dev),
                 trip_chi2=torch.zeros((n_t, nt), dtype=torch.float32, device=dev))
        b = self.batch_struct(packed, states, n_events)
        lf_debug_triplets(self.ctx, b, _ptr(d["win_count"]), _ptr(d["n_trip"]), _ptr(d["trip"]),
                          _ptr(d["trip_chi2"]), _stream(stream))
        return d

    def validate(self, packed: dict, states, n_events: int, stream=None) -> None:
        """lf_validate_batch: raises LFError naming the first broken input
        convention (offsets, x order inside a bucket, coarse index)."""
        lf_validate_batch(self.ctx, self.batch_struct(packed, states, n_events), _stream(stream))

    def status(self, stream=None) -> int:
        return lf_sync_status(self.ctx, _stream(stream))

    def reserve(self, n_events: int, n_hits: int, n_tracks: int, tuning: Optional[dict] = None) -> None:
        """Size the persistent form's scratch for batches up to these sizes."""
        tu = tuning_struct(tuning)
        lf_reserve(self.ctx, n_events, n_hits, n_tracks, tu)

    @staticmethod
    def _hptr(t: torch.Tensor):
        if t.is_cuda:
            raise ValueError("expected a host tensor")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return _P(t.data_ptr()) if t.numel() else None

    @staticmethod
    def alloc_host_output(n_tracks: int, pin: bool = True) -> dict:
        e = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=pin)
        return dict(found=e(n_tracks, torch.uint8), nhits=e(n_tracks, torch.uint8),
                    hit_idx=e((n_tracks, NL), torch.int32), state=e((n_tracks, 6), torch.float32),
                    quality=e(n_tracks, torch.float32))

    def process_host(self, batch, out: Optional[dict] = None, tuning: Optional[dict] = None,
                     chunk_hits: int = 0) -> dict:
        """End to end on host tensors (pinned for full speed): copies in,
        pack, find, copies the per-track results out; hit_idx are raw
        indices of the input batch."""
        h = self._hptr
        n_t = int(batch.sx.numel())
        if out is None:
            out = self.alloc_host_output(n_t)
        hb = lf_host_batch(int(batch.n_events), int(batch.x.numel()), n_t, h(batch.raw_offsets), h(batch.x),
                           h(batch.z), h(batch.dxdy), h(batch.w), h(batch.plane), h(batch.trk_offsets), h(batch.sx),
                           h(batch.sy), h(batch.stx), h(batch.sty), h(batch.sqop))
        ho = lf_host_output(h(out["found"]), h(out["nhits"]), h(out["hit_idx"]), h(out["state"]), h(out["quality"]))
        tu = tuning_struct(tuning)
        lf_process_host(self.ctx, hb, ho, tu, int(chunk_hits))
        return out

    def run(self, raw, mode: str = "batched", tuning: Optional[dict] = None, stream=None):
        """pack + find for a batch whose tensors live on the GPU."""
        packed = self.pack(raw, stream)
        out = self.find(packed, raw, raw.n_events, mode, tuning, stream)
        return packed, out

    def process_slot(self, slot: "SlotBuffers", pool=None, tuning: Optional[dict] = None, stream=None) -> None:
        """lf_process_slot on a slot's buffers: the batch whose event count is
        in slot.n_dev (and offsets in slot.raw_offsets / slot.trk_offsets);
        pool (an object with device x, z, dxdy, w, plane, sx, sy, stx, sty,
        sqop) is the gather source, read through slot.hit_src / slot.trk_src."""
        raw, pk, b, o = slot.structs(pool)
        g = None
        if pool is not None:
            g = lf_gather(_ptr(slot.hit_src), _ptr(slot.trk_src), _ptr(pool.sx), _ptr(pool.sy), _ptr(pool.stx),
                          _ptr(pool.sty), _ptr(pool.sqop))
        lf_process_slot(self.ctx, raw, pk, b, g, slot.n_dev.data_ptr(), o, tuning_struct(tuning), _stream(stream))

    def graph_count(self) -> int:
        return lf_graph_count(self.ctx)


class SlotBuffers:
    """Device buffers of one slot of lf_process_slot, of fixed capacity:
    offsets, states, packed hits, outputs, the event count (n_dev) and the
    gather indices; raw hit arrays too unless the slot gathers from a pool."""

    def __init__(self, max_events: int, max_hits: int, max_tracks: int, device, own_raw: bool = True):
        e = lambda n, dt: torch.empty(max(int(n), 1), dtype=dt, device=device)
        self.max_events, self.max_hits, self.max_tracks = int(max_events), int(max_hits), int(max_tracks)
        # the per-batch values in one int32 block (one copy from the host per
        # batch): event count, raw and track offsets, gather sources
        self.meta = torch.zeros(self.meta_size(self.max_events), dtype=torch.int32, device=device)
        self.n_dev, self.raw_offsets, self.trk_offsets, self.hit_src, self.trk_src = self.meta_views(self.meta)
        self.raw = None
        if own_raw:
            self.raw = dict(x=e(max_hits, torch.float32), z=e(max_hits, torch.float32),
                            dxdy=e(max_hits, torch.float32), w=e(max_hits, torch.float32),
                            plane=e(max_hits, torch.uint8))
        self.states = dict(sx=e(max_tracks, torch.float32), sy=e(max_tracks, torch.float32),
                           stx=e(max_tracks, torch.float32), sty=e(max_tracks, torch.float32),
                           sqop=e(max_tracks, torch.float32))
        self.packed = dict(hit_offsets=e(NB * max_events + 1, torch.int32), x=e(max_hits, torch.float32),
                           z=e(max_hits, torch.float32), dxdy=e(max_hits, torch.float32),
                           w=e(max_hits, torch.float32), layer=e(max_hits, torch.uint8),
                           perm=e(max_hits, torch.int32), x_coarse=e(coarse_count(max_hits), torch.float32))
        self.out = Tracker.alloc_output(self.max_tracks, self.max_events, device)

    @staticmethod
    def meta_size(max_events: int) -> int:
        return 1 + 2 * (max_events + 1) + 2 * max(max_events, 1)

    def meta_views(self, meta: torch.Tensor):
        """(n_dev, raw_offsets, trk_offsets, hit_src, trk_src) views of a
        block of meta_size int32 values (device, or a host staging copy)."""
        c = self.max_events
        a, b, d = 1 + (c + 1), 1 + 2 * (c + 1), 1 + 2 * (c + 1) + max(c, 1)
        return meta[0:1], meta[1:a], meta[a:b], meta[b:d], meta[d:d + max(c, 1)]

    def structs(self, pool=None):
        src = pool if pool is not None else SimpleRaw(self.raw)
        raw = lf_raw_hits(self.max_events, self.max_hits, _ptr(self.raw_offsets), _ptr(src.x), _ptr(src.z),
                          _ptr(src.dxdy), _ptr(src.w), _ptr(src.plane))
        pk = self.packed
        packed = lf_packed(_ptr(pk["hit_offsets"]), _ptr(pk["x"]), _ptr(pk["z"]), _ptr(pk["dxdy"]), _ptr(pk["w"]),
                           _ptr(pk["layer"]), _ptr(pk["perm"]), _ptr(pk["x_coarse"]))
        st = self.states
        b = lf_batch(self.max_events, self.max_hits, self.max_tracks, _ptr(pk["hit_offsets"]), _ptr(pk["x"]),
                     _ptr(pk["z"]), _ptr(pk["dxdy"]), _ptr(pk["w"]), _ptr(self.trk_offsets), _ptr(st["sx"]),
                     _ptr(st["sy"]), _ptr(st["stx"]), _ptr(st["sty"]), _ptr(st["sqop"]), _ptr(pk["x_coarse"]))
        return raw, packed, b, Tracker.output_struct(self.out)


class SimpleRaw:
    """Attribute view of a dict of raw hit arrays."""

    def __init__(self, d: dict):
        self.__dict__.update(d)


def numa_node_cpus() -> dict:
    """NUMA node -> CPU ids of this host that the process may run on (from
    /sys; empty when the host reports no nodes)."""
    import glob
    allowed = os.sched_getaffinity(0)
    out = {}
    for path in sorted(glob.glob("/sys/devices/system/node/node[0-9]*/cpulist")):
        node = int(path.split("/node")[-1].split("/")[0])
        cpus = set()
        for part in open(path).read().strip().split(","):
            if not part:
                continue
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        if cpus & allowed:
            out[node] = sorted(cpus & allowed)
    return out
