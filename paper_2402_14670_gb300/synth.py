"""Seeded synthetic SciFi events: the inputs of the forward-tracking path.

This module simulates the detector only. It draws particles, propagates them
with the trajectory model of the paper (Sec. "Propagation of tracks in LHCb's
magnetic field", Eq. trackfitmodel, with the linear pT kick of Eq. pt_kick at
the magnet centre), records smeared hits in the twelve x-u-v-x layers, adds
uniform noise and writes the upstream track states.  It performs none of the
reconstruction: no window, search, fit or selection happens here.  Both the
CUDA path and the CPU oracle consume what it produces.

Geometry and occupancies follow the five synthetic workloads of the paper's
stand-in benchmark (tiny single event, minimum-bias batch, uneven batch,
served stream, high occupancy); see ``CONFIGS``.

Everything is a torch tensor on the requested device.  Random numbers come
from a ``torch.Generator`` seeded per (workload seed, block of events), so a
workload is reproducible for a given device and event count.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional

import numpy as np
import torch

N_LAYERS = 12
N_ZONES = 2
N_BUCKETS = N_LAYERS * N_ZONES  # (zone, layer) buckets per event

# z of the 12 SciFi layers (mm), three x-u-v-x stations T1..T3.
LAYER_Z = (7826.0, 7896.0, 7966.0, 8036.0,
           8508.0, 8578.0, 8648.0, 8718.0,
           9193.0, 9263.0, 9333.0, 9403.0)
LAYER_KIND = ("x", "u", "v", "x") * 3
STEREO_DEG = 5.0


def _f32(v: float) -> float:
    """Round a Python float to the nearest binary32 value."""
    return float(np.float32(v))


@dataclasses.dataclass
class Geometry:
    """Detector and field constants, all representable in binary32."""
    z: tuple = LAYER_Z
    dxdy: tuple = None            # 0 for x layers, +tan(5 deg) for u, -tan(5 deg) for v
    z_state: float = 2700.0       # z of the upstream (VELO-UT) state
    z_magnet: float = 5200.0      # kick plane
    z_ref: float = 8520.0         # reference plane of the T-station model
    kappa: float = 1.2            # GeV rad: slope kick = polarity*kappa*q/p
    gamma: float = 2.4e-9         # GeV/mm^2: curvature c = polarity*gamma*q/p
    dratio: float = 4e-4          # 1/mm
    polarity: int = 1             # +1 MagUp, -1 MagDown

    def __post_init__(self):
        if self.dxdy is None:
            t = math.tan(math.radians(STEREO_DEG))
            self.dxdy = tuple(0.0 if k == "x" else (t if k == "u" else -t) for k in LAYER_KIND)
        self.z = tuple(_f32(v) for v in self.z)
        self.dxdy = tuple(_f32(v) for v in self.dxdy)
        for f in ("z_state", "z_magnet", "z_ref", "kappa", "gamma", "dratio"):
            setattr(self, f, _f32(getattr(self, f)))


@dataclasses.dataclass
class EventConfig:
    name: str
    n_events: int
    seed: int
    n_in: tuple                      # ("fixed", n) | ("poisson", mean) | ("negbin", mean, r, lo, hi) | ("uniform", lo, hi)
    match_frac: float = 0.7          # fraction of input states that belong to a particle with SciFi hits
    extra: tuple = ("none",)         # ("poisson", mean) | ("per_track", kmin, kmax, hits_per_particle) | ("signal", hits, hits_per_particle)
    noise: tuple = ("frac", 0.3)     # ("per_layer", n) | ("frac", f): noise hits = f/(1-f) * signal hits
    p_min: float = 3.0               # GeV
    p_max: float = 50.0
    tx_max: float = 0.25
    ty_max: float = 0.2
    sigma: float = 0.08              # mm, in the measured coordinate
    efficiency: float = 0.98
    qop_smear: float = 0.15          # relative smear of the input q/p
    x_acc: float = 3000.0
    y_acc: float = 2500.0


CONFIGS: Dict[int, EventConfig] = {
    0: EventConfig("tiny single event", 1, 1, ("fixed", 20), match_frac=1.0,
                   extra=("none",), noise=("per_layer", 200)),
    1: EventConfig("minimum-bias batch", 1000, 2, ("poisson", 60.0),
                   extra=("poisson", 440.0), noise=("frac", 0.3)),
    2: EventConfig("uneven batch", 100_000, 3, ("negbin", 80.0, 2.0, 1, 400),
                   extra=("per_track", 100.0, 150.0, 11.6), noise=("frac", 0.3)),
    3: EventConfig("served stream", 100_000, 4, ("negbin", 80.0, 2.0, 1, 400),
                   extra=("per_track", 100.0, 150.0, 11.6), noise=("frac", 0.3)),
    4: EventConfig("high occupancy", 20_000, 5, ("uniform", 300, 600),
                   extra=("signal", 12500.0, 11.0), noise=("frac", 0.5), p_min=1.5),
}


@dataclasses.dataclass
class EventBatch:
    """A batch of raw events (hits unsorted inside each event) plus truth."""
    n_events: int
    raw_offsets: torch.Tensor     # int32 [n_events+1]
    x: torch.Tensor               # float32 measured coordinate (x - y*dxdy)
    z: torch.Tensor               # float32
    dxdy: torch.Tensor            # float32
    w: torch.Tensor               # float32 weight 1/sigma^2
    plane: torch.Tensor           # uint8 zone*12 + layer (zone 1 = y >= 0)
    trk_offsets: torch.Tensor     # int32 [n_events+1]
    sx: torch.Tensor              # float32 upstream state at z_state
    sy: torch.Tensor
    stx: torch.Tensor
    sty: torch.Tensor
    sqop: torch.Tensor
    # truth (None when generated with truth=False)
    hit_mcp: Optional[torch.Tensor] = None     # int32 particle id, -1 noise
    hit_x64: Optional[torch.Tensor] = None     # float64 unsmeared measured coordinate
    trk_mcp: Optional[torch.Tensor] = None     # int32 particle id of each input state, -1 if none
    mcp: Optional[Dict[str, torch.Tensor]] = None  # per particle float64 truth

    @property
    def n_hits(self) -> int:
        return int(self.x.numel())

    @property
    def n_tracks(self) -> int:
        return int(self.sx.numel())

    def to(self, device) -> "EventBatch":
        kw = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if isinstance(v, torch.Tensor):
                v = v.to(device)
            elif isinstance(v, dict):
                v = {k: t.to(device) for k, t in v.items()}
            kw[f.name] = v
        return EventBatch(**kw)

    def select_events(self, idx) -> "EventBatch":
        """A new batch made of the listed events, in the listed order."""
        idx = [int(i) for i in idx]
        ro = self.raw_offsets.cpu().numpy().astype(np.int64)
        to = self.trk_offsets.cpu().numpy().astype(np.int64)
        dev = self.x.device
        hsel = np.concatenate([np.arange(ro[e], ro[e + 1]) for e in idx]) if idx else np.zeros(0, np.int64)
        tsel = np.concatenate([np.arange(to[e], to[e + 1]) for e in idx]) if idx else np.zeros(0, np.int64)
        hs = torch.from_numpy(hsel).to(dev)
        ts = torch.from_numpy(tsel).to(dev)
        nh = np.array([ro[e + 1] - ro[e] for e in idx], np.int64)
        nt = np.array([to[e + 1] - to[e] for e in idx], np.int64)
        mk = lambda n: torch.from_numpy(np.concatenate([[0], np.cumsum(n)]).astype(np.int32)).to(dev)
        g = lambda t: None if t is None else t[hs]
        gt = lambda t: None if t is None else t[ts]
        return EventBatch(len(idx), mk(nh), self.x[hs], self.z[hs], self.dxdy[hs], self.w[hs],
                          self.plane[hs], mk(nt), self.sx[ts], self.sy[ts], self.stx[ts],
                          self.sty[ts], self.sqop[ts], g(self.hit_mcp), g(self.hit_x64),
                          gt(self.trk_mcp), self.mcp)

    def pin_memory(self) -> "EventBatch":
        kw = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if isinstance(v, torch.Tensor) and f.name not in ("hit_mcp", "hit_x64", "trk_mcp"):
                v = v.pin_memory()
            kw[f.name] = v
        return EventBatch(**kw)


def trajectory(tx, ty, qop, geo: Optional[Geometry] = None):
    """Simulated particle from the origin with VELO slopes (tx, ty) and q/p:
    returns (x, y, x_measured) at the 12 layers in binary64, where
    x_measured = x - y*dxdy is the coordinate a (stereo) layer records."""
    geo = geo or Geometry()
    tx = np.asarray(tx, np.float64)[..., None]
    ty = np.asarray(ty, np.float64)[..., None]
    qop = np.asarray(qop, np.float64)[..., None]
    z = np.asarray(geo.z, np.float64)
    dxdy = np.asarray(geo.dxdy, np.float64)
    pol = float(geo.polarity)
    txf = tx + pol * geo.kappa * qop
    cc = pol * geo.gamma * qop
    dz = z - geo.z_ref
    x = tx * geo.z_magnet + txf * (z - geo.z_magnet) + cc * (dz * dz * (1.0 + geo.dratio * dz))
    y = ty * z
    return x, y, x - y * dxdy


def state_of(tx, ty, qop, geo: Optional[Geometry] = None):
    """Upstream state (x, y, tx, ty, q/p) at z_state of a particle from the origin."""
    geo = geo or Geometry()
    return (tx * geo.z_state, ty * geo.z_state, tx, ty, qop)


def truth_params(tx, ty, qop, geo: Optional[Geometry] = None):
    """Track parameters at z_ref: (x, y, tx, ty, c, q/p) in binary64."""
    geo = geo or Geometry()
    pol = float(geo.polarity)
    txf = tx + pol * geo.kappa * qop
    return (tx * geo.z_magnet + txf * (geo.z_ref - geo.z_magnet), ty * geo.z_ref, txf, ty,
            pol * geo.gamma * qop, qop)


def _block_seed(seed: int, block: int) -> int:
    # splitmix64 of (seed, block): independent streams per block
    v = (seed * 0x9E3779B97F4A7C15 + block + 1) & 0xFFFFFFFFFFFFFFFF
    v ^= v >> 30
    v = (v * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    v ^= v >> 27
    v = (v * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    v ^= v >> 31
    return v & 0x7FFFFFFFFFFFFFFF


def _draw_counts(spec, n, g, dev):
    kind = spec[0]
    if kind == "fixed":
        return torch.full((n,), int(spec[1]), dtype=torch.int64, device=dev)
    if kind == "poisson":
        lam = torch.full((n,), float(spec[1]), dtype=torch.float64, device=dev)
        return torch.poisson(lam, generator=g).to(torch.int64)
    if kind == "negbin":
        mean, r, lo, hi = spec[1], spec[2], spec[3], spec[4]
        # Gamma-Poisson mixture: lambda ~ Gamma(r, mean/r)
        gam = torch._standard_gamma(torch.full((n,), float(r), dtype=torch.float64, device=dev),
                                    generator=g) * (mean / r)
        k = torch.poisson(gam, generator=g).to(torch.int64)
        return k.clamp(int(lo), int(hi))
    if kind == "uniform":
        lo, hi = int(spec[1]), int(spec[2])
        return torch.randint(lo, hi + 1, (n,), generator=g, device=dev, dtype=torch.int64)
    raise ValueError(spec)


def _generate_block(cfg: EventConfig, geo: Geometry, n_ev: int, seed: int, dev, truth: bool):
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    f64 = torch.float64
    U = lambda *s: torch.rand(*s, generator=g, device=dev, dtype=f64)
    N = lambda *s: torch.randn(*s, generator=g, device=dev, dtype=f64)

    n_in = _draw_counts(cfg.n_in, n_ev, g, dev)
    T = int(n_in.sum())
    trk_ev = torch.repeat_interleave(torch.arange(n_ev, device=dev), n_in)
    matched = U(T) < cfg.match_frac
    n_matched_ev = torch.zeros(n_ev, dtype=torch.int64, device=dev).index_add_(0, trk_ev, matched.to(torch.int64))

    kind = cfg.extra[0]
    if kind == "none":
        n_extra = torch.zeros(n_ev, dtype=torch.int64, device=dev)
    elif kind == "poisson":
        n_extra = torch.poisson(torch.full((n_ev,), float(cfg.extra[1]), dtype=f64, device=dev), generator=g).to(torch.int64)
    elif kind == "per_track":
        k = cfg.extra[1] + (cfg.extra[2] - cfg.extra[1]) * U(n_ev)
        total = torch.round(k * n_in.to(f64) / cfg.extra[3]).to(torch.int64)
        n_extra = (total - n_matched_ev).clamp_min(0)
    elif kind == "signal":
        total = torch.poisson(torch.full((n_ev,), cfg.extra[1] / cfg.extra[2], dtype=f64, device=dev), generator=g).to(torch.int64)
        n_extra = (total - n_matched_ev).clamp_min(0)
    else:
        raise ValueError(cfg.extra)
    E = int(n_extra.sum())
    extra_ev = torch.repeat_interleave(torch.arange(n_ev, device=dev), n_extra)

    # kinematics of every input state and every extra particle
    K = T + E
    lp = math.log(cfg.p_min) + (math.log(cfg.p_max) - math.log(cfg.p_min)) * U(K)
    p = torch.exp(lp)
    q = torch.where(U(K) < 0.5, -1.0, 1.0).to(f64)
    tx = (2.0 * U(K) - 1.0) * cfg.tx_max
    ty = (2.0 * U(K) - 1.0) * cfg.ty_max
    qop = q / p

    # particles with SciFi hits: matched input states, then the extra particles
    part_sel = torch.cat([torch.nonzero(matched).flatten(), torch.arange(T, K, device=dev)])
    part_ev = torch.cat([trk_ev[matched], extra_ev])
    P = int(part_sel.numel())
    pq, ptx, pty = qop[part_sel], tx[part_sel], ty[part_sel]
    pol = float(geo.polarity)
    txf = ptx + pol * geo.kappa * pq
    cc = pol * geo.gamma * pq
    xmag = ptx * geo.z_magnet

    z = torch.tensor(geo.z, dtype=f64, device=dev)
    dxdy = torch.tensor(geo.dxdy, dtype=f64, device=dev)
    dz = z - geo.z_ref
    xz = xmag[:, None] + txf[:, None] * (z - geo.z_magnet)[None, :] + cc[:, None] * (dz * dz * (1.0 + geo.dratio * dz))[None, :]
    yz = pty[:, None] * z[None, :]
    xm = xz - yz * dxdy[None, :]
    keep = (xz.abs() < cfg.x_acc) & (yz.abs() < cfg.y_acc) & (U(P, N_LAYERS) < cfg.efficiency)
    smeared = xm + cfg.sigma * N(P, N_LAYERS)
    pi, li = torch.nonzero(keep, as_tuple=True)
    sig_x = smeared[pi, li]
    sig_x64 = xm[pi, li]
    sig_layer = li
    sig_zone = (yz[pi, li] >= 0).to(torch.int64)
    sig_ev = part_ev[pi]
    sig_mcp = pi
    n_sig_ev = torch.zeros(n_ev, dtype=torch.int64, device=dev).index_add_(0, sig_ev, torch.ones_like(sig_ev))

    # uniform noise hits
    if cfg.noise[0] == "per_layer":
        n_noise = torch.full((n_ev,), int(cfg.noise[1]) * N_LAYERS, dtype=torch.int64, device=dev)
    else:
        f = float(cfg.noise[1])
        n_noise = torch.round(n_sig_ev.to(f64) * (f / (1.0 - f))).to(torch.int64)
    Nn = int(n_noise.sum())
    noise_ev = torch.repeat_interleave(torch.arange(n_ev, device=dev), n_noise)
    if cfg.noise[0] == "per_layer":
        per = int(cfg.noise[1])
        noise_layer = torch.arange(N_LAYERS, device=dev).repeat_interleave(per).repeat(n_ev)
    else:
        noise_layer = torch.randint(0, N_LAYERS, (Nn,), generator=g, device=dev)
    noise_zone = (U(Nn) < 0.5).to(torch.int64)
    noise_x = (2.0 * U(Nn) - 1.0) * cfg.x_acc

    h_ev = torch.cat([sig_ev, noise_ev])
    h_x64 = torch.cat([sig_x64, noise_x])
    h_x = torch.cat([sig_x, noise_x])
    h_layer = torch.cat([sig_layer, noise_layer])
    h_zone = torch.cat([sig_zone, noise_zone])
    h_mcp = torch.cat([sig_mcp, torch.full((Nn,), -1, dtype=torch.int64, device=dev)])

    # event-major order, random order inside each event
    rnd = torch.randint(0, 1 << 31, (h_ev.numel(),), generator=g, device=dev, dtype=torch.int64)
    order = torch.argsort(h_ev * (1 << 31) + rnd)
    h_ev, h_x, h_x64, h_layer, h_zone, h_mcp = (t[order] for t in (h_ev, h_x, h_x64, h_layer, h_zone, h_mcp))
    nh_ev = torch.zeros(n_ev, dtype=torch.int64, device=dev).index_add_(0, h_ev, torch.ones_like(h_ev))

    zf = torch.tensor(geo.z, dtype=torch.float32, device=dev)
    df = torch.tensor(geo.dxdy, dtype=torch.float32, device=dev)
    w = 1.0 / (cfg.sigma * cfg.sigma) if cfg.sigma > 0 else 1.0 / (0.08 * 0.08)
    out = dict(
        nh=nh_ev, nt=n_in,
        x=h_x.to(torch.float32), z=zf[h_layer], dxdy=df[h_layer],
        w=torch.full((h_x.numel(),), w, dtype=torch.float32, device=dev),
        plane=(h_zone * N_LAYERS + h_layer).to(torch.uint8),
    )
    # upstream states of every input track at z_state (straight line from the origin)
    zs = geo.z_state
    smear = 1.0 + cfg.qop_smear * N(T) if cfg.qop_smear > 0 else torch.ones(T, dtype=f64, device=dev)
    smear = smear.clamp_min(0.1)
    out.update(sx=(tx[:T] * zs).to(torch.float32), sy=(ty[:T] * zs).to(torch.float32),
               stx=tx[:T].to(torch.float32), sty=ty[:T].to(torch.float32),
               sqop=(qop[:T] * smear).to(torch.float32))
    if truth:
        trk_mcp = torch.full((T,), -1, dtype=torch.int64, device=dev)
        trk_mcp[matched] = torch.arange(int(matched.sum()), device=dev)
        out.update(hit_mcp=h_mcp, hit_x64=h_x64, trk_mcp=trk_mcp,
                   mcp=dict(qop=pq, tx=ptx, ty=pty, txf=txf, c=cc,
                            xref=xmag + txf * (geo.z_ref - geo.z_magnet), yref=pty * geo.z_ref,
                            event=part_ev, nhits=keep.sum(1)))
        out["P"] = P
    return out


def generate(config, n_events: Optional[int] = None, device="cpu", truth: bool = True,
             geometry: Optional[Geometry] = None, block_events: int = 4096, **overrides) -> EventBatch:
    """Generate a batch of raw events for workload ``config`` (an int key of
    ``CONFIGS`` or an ``EventConfig``).  ``overrides`` replace config fields
    (e.g. ``sigma=0.0, efficiency=1.0, noise=("per_layer", 0)`` for the
    noise-free closed-form case)."""
    cfg = CONFIGS[config] if isinstance(config, int) else config
    if overrides:
        cfg = dataclasses.replace(cfg, **overrides)
    geo = geometry or Geometry()
    n_events = cfg.n_events if n_events is None else int(n_events)
    dev = torch.device(device)
    parts = []
    for b, start in enumerate(range(0, max(n_events, 1), block_events)):
        nb = min(block_events, n_events - start)
        if nb <= 0:
            break
        parts.append(_generate_block(cfg, geo, nb, _block_seed(cfg.seed, b), dev, truth))
    if not parts:
        z32 = torch.zeros(1, dtype=torch.int32, device=dev)
        e = torch.zeros(0, dtype=torch.float32, device=dev)
        return EventBatch(0, z32, e, e, e, e, torch.zeros(0, dtype=torch.uint8, device=dev), z32.clone(), e, e, e, e, e)

    cat = lambda k: torch.cat([pp[k] for pp in parts])
    nh = cat("nh")
    nt = cat("nt")
    off = lambda n: torch.cat([torch.zeros(1, dtype=torch.int64, device=dev), torch.cumsum(n, 0)]).to(torch.int32)
    if int(nh.sum()) >= 2**31 - 1:
        raise ValueError("batch too large for int32 hit offsets")
    batch = EventBatch(n_events, off(nh), cat("x"), cat("z"), cat("dxdy"), cat("w"), cat("plane"),
                       off(nt), cat("sx"), cat("sy"), cat("stx"), cat("sty"), cat("sqop"))
    if truth:
        mc_off, tr, hm = 0, [], []
        for pp in parts:
            tr.append(torch.where(pp["trk_mcp"] >= 0, pp["trk_mcp"] + mc_off, pp["trk_mcp"]))
            hm.append(torch.where(pp["hit_mcp"] >= 0, pp["hit_mcp"] + mc_off, pp["hit_mcp"]))
            mc_off += pp["P"]
        batch.trk_mcp = torch.cat(tr).to(torch.int32)
        batch.hit_mcp = torch.cat(hm).to(torch.int32)
        batch.hit_x64 = cat("hit_x64")
        ev_off, mcs = 0, []
        for bi, pp in enumerate(parts):
            m = dict(pp["mcp"])
            m["event"] = m["event"] + ev_off
            ev_off += int(pp["nh"].numel())
            mcs.append(m)
        batch.mcp = {k: torch.cat([m[k] for m in mcs]) for k in mcs[0]}
    return batch


def geometry_dict(geo: Optional[Geometry] = None) -> dict:
    geo = geo or Geometry()
    return dataclasses.asdict(geo)
