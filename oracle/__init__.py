"""CPU oracle of the Looking Forward path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does.

It wraps ``lf_oracle.c`` (plain single-threaded C, binary32 without
contraction, plus a binary64 refit) through ctypes.  ``build()`` compiles it
with gcc; nothing here is shared with the CUDA path.

Parameter defaults are the "Forward" column of the paper's Table tolerances,
Table C_nhits and the constants of Sec. "Defining the search windows" and
"Triplet Seeding"; the readings for what the paper leaves open are noted
beside each value.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lf_oracle.c")
HDR = os.path.join(HERE, "lf_oracle.h")
LIB = os.path.join(HERE, "liblf_oracle.so")
NL = 12
NB = 24
MAX_TRIP = 32

# ---------------------------------------------------------------- defaults

#: geometry of the synthetic detector: layer z (x-u-v-x stations), stereo
#: slopes +-tan(5 deg), kick plane and reference plane (z_ref = 8520 mm,
#: Sec. "Extending triplets to other layers").
def default_geometry() -> dict:
    t = float(np.float32(np.tan(np.radians(5.0))))
    kinds = ("x", "u", "v", "x") * 3
    return dict(
        z=[7826.0, 7896.0, 7966.0, 8036.0, 8508.0, 8578.0, 8648.0, 8718.0,
           9193.0, 9263.0, 9333.0, 9403.0],
        dxdy=[0.0 if k == "x" else (t if k == "u" else -t) for k in kinds],
        z_state=2700.0, z_magnet=5200.0, z_ref=8520.0,
        kappa=1.2, gamma=2.4e-9, dratio=4e-4, polarity=1)


#: Table poly_tol: c0..c7 of Eq. tol_noUT.
TOL_C = (4824.3, 426.3, 7071.1, 12080.4, 14077.8, 13909.3, 9315.3, 3209.5)


#: "Forward" column of Table tolerances and Table C_nhits.
def default_params(paper_K: bool = False) -> dict:
    return dict(
        xtol_c=150.0, xtol_p=2000.0,      # x_tol = 150 mm + 2000 mm GeV / p
        x_asym=100.0,                      # magnet asymmetry term
        uv_tol=800.0,                      # u/v window half width
        n_hits_window=32, n_triplets=12, min_hits=9,
        # K_x1: the paper's values are sagitta corrections for the real field;
        # the synthetic detector has no field in the T stations, so 1.0 is the
        # default and paper_K=True selects the printed constants.
        K_first=1.00177513 if paper_K else 1.0,
        K_last=1.00142634 if paper_K else 1.0,
        p_bend=5.0,                        # bending-sign filter below 5 GeV
        # magnet tolerance "from 8 to 40 mm" as a function of p and t_x^doublet:
        # clamp(8 + 96/p + 10|t_x|, 8, 40) mm (the paper prints no formula)
        magtol_min=8.0, magtol_max=40.0, magtol_c=96.0, magtol_tx=10.0,
        T_triplet=8.0, T_x=2.0,
        T_uv_scale=50.0, T_uv_min=2.0,     # T_uv = max(2, 50 (|t_x| + |t_y|))
        T_ty=0.02, T_y=800.0, T_Q=0.5,
        C_n=[5.0, 1.0, 0.8, 0.5],
        # Sec. "No-UT tuning" (used when no_ut = 1): assumed momentum from
        # p >= 5 GeV or pT >= 1 GeV, whichever is tighter; 5 mm overlap of
        # the two one-sided windows; c0..c7 of Table poly_tol
        no_ut=0, p_min=5.0, pt_min=1.0, x_overlap=5.0,
        tol_c=list(TOL_C),
        # Sec. "Calculation of momentum and track states": 0 = linear kick;
        # 1 = Eq. pt_kick with the polynomial field integral (coefficients
        # from a fit on toy tracks, qop_c[i][j])
        qop_poly=0, qop_c=[[0.0] * 10 for _ in range(5)])


#: "Forward no-UT" column of Table tolerances with the no-UT window and
#: seeding constants of Sec. "No-UT tuning": 1200 mm u/v tolerance, a fixed
#: 10 mm tolerance at the magnet, 64 hits per window, 20 triplets.
def no_ut_params() -> dict:
    p = default_params()
    p.update(no_ut=1, uv_tol=1200.0, n_hits_window=64, n_triplets=20,
             magtol_min=10.0, magtol_max=10.0, magtol_c=0.0, magtol_tx=0.0,
             T_triplet=2.0, T_x=0.5,
             T_uv_scale=15.0, T_uv_min=0.5,    # T_uv = max(T_x, 15 (|t_x| + |t_y|))
             T_ty=0.003, T_y=800.0, T_Q=0.5)
    return p


# ------------------------------------------------------------------ ctypes

class _Geo(C.Structure):
    _fields_ = [("z", C.c_float * NL), ("dxdy", C.c_float * NL),
                ("z_state", C.c_float), ("z_magnet", C.c_float), ("z_ref", C.c_float),
                ("kappa", C.c_float), ("gamma", C.c_float), ("dratio", C.c_float),
                ("polarity", C.c_int32)]


class _Par(C.Structure):
    _fields_ = [("xtol_c", C.c_float), ("xtol_p", C.c_float), ("x_asym", C.c_float),
                ("uv_tol", C.c_float), ("n_hits_window", C.c_int32), ("n_triplets", C.c_int32),
                ("min_hits", C.c_int32), ("K_first", C.c_float), ("K_last", C.c_float),
                ("p_bend", C.c_float), ("magtol_min", C.c_float), ("magtol_max", C.c_float),
                ("magtol_c", C.c_float), ("magtol_tx", C.c_float), ("T_triplet", C.c_float),
                ("T_x", C.c_float), ("T_uv_scale", C.c_float), ("T_uv_min", C.c_float),
                ("T_ty", C.c_float), ("T_y", C.c_float), ("T_Q", C.c_float),
                ("C_n", C.c_float * 4), ("no_ut", C.c_int32), ("p_min", C.c_float),
                ("pt_min", C.c_float), ("x_overlap", C.c_float), ("tol_c", C.c_float * 8),
                ("qop_poly", C.c_int32), ("qop_c", (C.c_float * 10) * 5)]


_P = C.c_void_p
_OUT_FIELDS = ["found", "nhits", "hit_idx", "state", "quality", "win_begin", "win_count",
               "win_xmin", "win_xmax", "win_centre", "n_trip", "trip", "trip_chi2",
               "cand_status", "cand_q", "state64"]


class _Out(C.Structure):
    _fields_ = [(f, _P) for f in _OUT_FIELDS]


_lock = threading.Lock()


def _compile(src_path: str, out_path: str, extra=()) -> None:
    tmp = out_path + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
           "-I", HERE, "-fPIC", "-shared", *extra, "-o", tmp, src_path, "-lpthread", "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out_path)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary32 without contraction)."""
    with _lock:
        stale = (not os.path.exists(LIB) or
                 os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)))
        if force or stale:
            _compile(SRC, LIB)
    return LIB


def _bind(path: str):
    lib = C.CDLL(path)
    lib.lfo_pack.restype = C.c_int
    lib.lfo_pack_mt.restype = C.c_int
    lib.lfo_find_tracks.restype = C.c_int
    lib.lfo_find_tracks_mt.restype = C.c_int
    lib.lfo_compact.restype = C.c_int32
    return lib


def _geo(g: dict) -> _Geo:
    s = _Geo()
    s.z[:] = [float(v) for v in g["z"]]
    s.dxdy[:] = [float(v) for v in g["dxdy"]]
    for k in ("z_state", "z_magnet", "z_ref", "kappa", "gamma", "dratio"):
        setattr(s, k, float(g[k]))
    s.polarity = int(g["polarity"])
    return s


def _par(p: dict) -> _Par:
    s = _Par()
    for name, _ in _Par._fields_:
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


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P)


def _c(a, dt):
    return np.ascontiguousarray(np.asarray(a), dtype=dt)


# ------------------------------------------------------------------ API

def _alloc_out(n_trk: int, dumps: bool, n_sides: int = 1):
    nw = n_trk * n_sides * NL
    o = dict(found=np.zeros(n_trk, np.uint8), nhits=np.zeros(n_trk, np.uint8),
             hit_idx=np.zeros(n_trk * NL, np.int32), state=np.zeros(n_trk * 6, np.float32),
             quality=np.zeros(n_trk, np.float32))
    if dumps:
        o.update(win_begin=np.zeros(nw, np.int32), win_count=np.zeros(nw, np.int32),
                 win_xmin=np.zeros(nw, np.float32), win_xmax=np.zeros(nw, np.float32),
                 win_centre=np.zeros(nw, np.float32), n_trip=np.zeros(n_trk, np.int32),
                 trip=np.full(n_trk * MAX_TRIP * 4, -1, np.int32),
                 trip_chi2=np.zeros(n_trk * MAX_TRIP, np.float32),
                 cand_status=np.full(n_trk * MAX_TRIP, -1, np.int32),
                 cand_q=np.zeros(n_trk * MAX_TRIP, np.float32),
                 state64=np.zeros(n_trk * 6, np.float64))
    st = _Out()
    for f in _OUT_FIELDS:
        setattr(st, f, _ptr(o[f]) if f in o else None)
    return o, st


def _shape(o: dict, n_trk: int, n_sides: int = 1) -> dict:
    """Per-track views; window dumps are (n_trk, n_sides*12), side-major."""
    r = dict(o)
    r["hit_idx"] = o["hit_idx"].reshape(n_trk, NL)
    r["state"] = o["state"].reshape(n_trk, 6)
    if "win_begin" in o:
        for k in ("win_begin", "win_count", "win_xmin", "win_xmax", "win_centre"):
            r[k] = o[k].reshape(n_trk, n_sides * NL)
        r["trip"] = o["trip"].reshape(n_trk, MAX_TRIP, 4)
        r["trip_chi2"] = o["trip_chi2"].reshape(n_trk, MAX_TRIP)
        r["cand_status"] = o["cand_status"].reshape(n_trk, MAX_TRIP)
        r["cand_q"] = o["cand_q"].reshape(n_trk, MAX_TRIP)
        r["state64"] = o["state64"].reshape(n_trk, 6)
    return r


class Oracle:
    """The oracle bound to one compiled copy of ``lf_oracle.c``."""

    def __init__(self, lib_path: str):
        self.lib = _bind(lib_path)

    def pack(self, raw_offsets, x, z, dxdy, w, plane, n_threads: int = 1) -> dict:
        """Bucket and sort raw hits: returns hit_offsets [24*n_ev+1], the
        packed x, z, dxdy, w, layer and perm (packed index -> raw index)."""
        ro = _c(raw_offsets, np.int32)
        n_ev = ro.size - 1
        arrs = [_c(a, np.float32) for a in (x, z, dxdy, w)]
        pl = _c(plane, np.uint8)
        n = arrs[0].size
        ho = np.zeros(NB * n_ev + 1, np.int32)
        outs = [np.zeros(n, np.float32) for _ in range(4)]
        layer = np.zeros(n, np.uint8)
        perm = np.zeros(n, np.int32)
        if n_threads > 1:
            rc = self.lib.lfo_pack_mt(C.c_int32(n_ev), _ptr(ro), *[_ptr(a) for a in arrs], _ptr(pl), _ptr(ho),
                                      *[_ptr(a) for a in outs], _ptr(layer), _ptr(perm), C.c_int32(n_threads))
            ho[NB * n_ev] = ro[n_ev] if n_ev else 0
        else:
            rc = self.lib.lfo_pack(C.c_int32(n_ev), _ptr(ro), *[_ptr(a) for a in arrs], _ptr(pl), _ptr(ho),
                                   *[_ptr(a) for a in outs], _ptr(layer), _ptr(perm))
        if rc != 0:
            raise ValueError("lfo_pack failed (%d)" % rc)
        return dict(hit_offsets=ho, x=outs[0], z=outs[1], dxdy=outs[2], w=outs[3],
                    layer=layer, perm=perm)

    def find_tracks(self, packed: dict, states: dict, geometry: dict = None, params: dict = None,
                    x64=None, dumps: bool = True, n_threads: int = 1) -> dict:
        """Run the whole path on packed hits.  ``states`` holds trk_offsets
        and sx, sy, stx, sty, sqop.  Returns per-track outputs (and, single
        threaded, the stage dumps)."""
        g = _geo(geometry or default_geometry())
        params = params or default_params()
        n_sides = 2 if params.get("no_ut", 0) else 1
        p = _par(params)
        ho = _c(packed["hit_offsets"], np.int32)
        n_ev = (ho.size - 1) // NB
        hx, hz, hd, hw = (_c(packed[k], np.float32) for k in ("x", "z", "dxdy", "w"))
        to = _c(states["trk_offsets"], np.int32)
        s = [_c(states[k], np.float32) for k in ("sx", "sy", "stx", "sty", "sqop")]
        n_trk = s[0].size
        o, st = _alloc_out(n_trk, dumps and n_threads == 1, n_sides)
        if n_threads == 1:
            x64a = None if x64 is None else _c(x64, np.float64)
            rc = self.lib.lfo_find_tracks(C.byref(g), C.byref(p), C.c_int32(n_ev), _ptr(ho), _ptr(hx),
                                          _ptr(hz), _ptr(hd), _ptr(hw),
                                          None if x64a is None else _ptr(x64a), _ptr(to),
                                          *[_ptr(a) for a in s], C.byref(st))
        else:
            rc = self.lib.lfo_find_tracks_mt(C.byref(g), C.byref(p), C.c_int32(n_ev), _ptr(ho),
                                             _ptr(hx), _ptr(hz), _ptr(hd), _ptr(hw), _ptr(to),
                                             *[_ptr(a) for a in s], C.byref(st), C.c_int32(n_threads))
        if rc != 0:
            raise ValueError("lfo_find_tracks failed (%d)" % rc)
        return _shape(o, n_trk, n_sides)

    def compact(self, trk_offsets, found):
        to = _c(trk_offsets, np.int32)
        fd = _c(found, np.uint8)
        n_ev = to.size - 1
        oo = np.zeros(n_ev + 1, np.int32)
        ot = np.zeros(max(fd.size, 1), np.int32)
        n = self.lib.lfo_compact(C.c_int32(n_ev), _ptr(to), _ptr(fd), _ptr(oo), _ptr(ot))
        return oo, ot[:n]

    def run_batch(self, batch, geometry=None, params=None, dumps=True, use_x64=False,
                  n_threads=1) -> dict:
        """Pack + find + compact for an ``EventBatch`` (tensors on any device)."""
        t = lambda a: a.detach().cpu().numpy()
        pk = self.pack(t(batch.raw_offsets), t(batch.x), t(batch.z), t(batch.dxdy), t(batch.w),
                       t(batch.plane), n_threads=n_threads)
        states = dict(trk_offsets=t(batch.trk_offsets), sx=t(batch.sx), sy=t(batch.sy),
                      stx=t(batch.stx), sty=t(batch.sty), sqop=t(batch.sqop))
        x64 = None
        if use_x64 and batch.hit_x64 is not None:
            x64 = t(batch.hit_x64)[pk["perm"]]
        res = self.find_tracks(pk, states, geometry, params, x64=x64, dumps=dumps,
                               n_threads=n_threads)
        oo, ot = self.compact(states["trk_offsets"], res["found"])
        res.update(packed=pk, out_offsets=oo, out_trk=ot)
        return res


_default = None


def default() -> Oracle:
    """The oracle built from ``lf_oracle.c`` as committed."""
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def variant(src_text: str, workdir: str, name: str) -> Oracle:
    """Compile a modified copy of the oracle source (used by tests that plant
    a mistake in the oracle to show that the pins catch it)."""
    src = os.path.join(workdir, name + ".c")
    with open(src, "w") as f:
        f.write(src_text)
    lib = os.path.join(workdir, "lib" + name + ".so")
    _compile(src, lib)
    return Oracle(lib)


def source() -> str:
    with open(SRC) as f:
        return f.read()


def pack(*a, **k):
    return default().pack(*a, **k)


def find_tracks(*a, **k):
    return default().find_tracks(*a, **k)


def compact(*a, **k):
    return default().compact(*a, **k)


def run_batch(*a, **k):
    return default().run_batch(*a, **k)
