"""Serving loop: render / relight requests against resident scenes.

Requests of uneven resolution and sample count arrive over time (a Poisson
stream).  Meshes, their BVHs, textures and the probes' sampling tables stay
resident on the device.  A request runs the forward hot path — rasterised
G-buffer, Monte Carlo direct illumination (Sec. 3.1, 4.1), the BF16 U-Net
denoiser on c_d and c_s (Sec. 4.2) and the composite c = k_d D(c_d) + D(c_s)
— as libmcdi launches on one of a few CUDA streams.

Continuous batching: requests that arrive while others are on the GPU are
admitted as soon as a stream slot is free and their memory fits the HBM
budget (footprint counted per request from its resolution and spp); work of
admitted requests overlaps on the device.  The one-request-at-a-time mode runs
the same stream through one slot.  Every request carries its own Philox seed,
so its image does not depend on what else is in flight.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import mcdi
from .scenes import RenderRequest, split_spp


@dataclass
class _Resident:
    verts: torch.Tensor
    vnrm: torch.Tensor
    tris: torch.Tensor
    bvh: mcdi.Bvh
    tex_kd: torch.Tensor
    tex_korm: torch.Tensor
    cams: torch.Tensor
    uvmap: list


@dataclass
class _InFlight:
    req: RenderRequest
    event: torch.cuda.Event
    bytes: int
    slot: int


class _Slot:
    """Buffers of one request slot, allocated once at the largest request size:
    every request's tensors are views of their leading elements, so admission
    allocates nothing.  `view(res)` returns those views."""

    def __init__(self, dev, max_res: int, max_spp: int):
        P = max_res * max_res
        f4 = lambda n: torch.empty((n * P * 4,), device=dev)
        self.planes = {k: f4(n) for k, n in (("pos", 1), ("nrm", 1), ("kd", 1), ("korm", 1), ("terms", 2),
                                               ("kd_out", 1), ("den", 2), ("color", 1))}
        prm = mcdi.make_params(*split_spp(max_spp), seed=1)
        self.ws = mcdi._empty_bytes(mcdi.shade_workspace_size(1, max_res, max_res, prm), dev)
        self.rws = mcdi._empty_bytes(mcdi.raster_workspace_size(1, max_res, max_res), dev)
        self.acts = mcdi._empty_bytes(mcdi.denoise_sizes(2, max_res, max_res)[1], dev)
        self.cam = torch.empty((1, 14), device=dev)
        self.graphs = {}  # res -> CUDA graph of the denoiser and the composite at that size

    def view(self, r: int) -> dict:
        v = lambda k, n: self.planes[k][: n * r * r * 4].view(n, r, r, 4)
        gb = mcdi.GBuffer(v("pos", 1), v("nrm", 1), v("kd", 1), v("korm", 1))
        return dict(gb=gb, terms=v("terms", 2), kd_out=v("kd_out", 1), den=v("den", 2), color=v("color", 1))


class ServingEngine:
    """sides: the image sides requests may ask for (the graphs of the denoiser tail are
    captured for each at start-up); max_spp: the largest sample count."""

    def __init__(self, scene_list, probe_list, denoiser_params, n_slots: int = 4, hbm_budget: int = 8 << 30,
                 device="cuda", tau: float = 1.0, sides=tuple(range(128, 1025, 32)), max_spp: int = 64):
        mcdi.load()
        self.dev = torch.device(device)
        dev = self.dev
        t = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
        self.scenes = []
        for sc in scene_list:
            verts, tris = t(sc["verts"]), t(sc["tris"], torch.int32)
            bvh = mcdi.Bvh.allocate(tris.shape[0], dev).build(verts, tris)
            self.scenes.append(_Resident(verts, t(sc["vnrm"]), tris, bvh, t(sc["tex_kd"]), t(sc["tex_korm"]),
                                         t(sc["cams"]), [float(x) for x in sc["uvmap"]]))
        self.probes = [mcdi.Probe.allocate(t(env)).build() for env in probe_list]
        wb, _, _, n_params = mcdi.denoise_sizes(2, 64, 64)
        p = torch.as_tensor(denoiser_params, dtype=torch.float32, device=dev)
        assert p.numel() == n_params
        self.den_weights = torch.empty((wb + 255) // 256 * 256, dtype=torch.uint8, device=dev)
        mcdi.denoise_pack_weights(p, self.den_weights)
        self.err = torch.zeros(1, dtype=torch.int32, device=dev)
        self.n_slots = n_slots
        self.hbm_budget = hbm_budget
        self.tau = tau
        self.sides = tuple(sorted(set(int(x) for x in sides)))
        self.max_spp = max_spp
        self.streams = [torch.cuda.Stream(dev) for _ in range(n_slots)]
        self._lanes = {}
        self.slots = [_Slot(dev, max(self.sides), max_spp) for _ in range(n_slots)]
        self._footprints = {}
        torch.cuda.synchronize(dev)
        self._capture_tails()

    # ---- the scene-independent tail of a request: denoiser on c_d and c_s, composite
    def _tail(self, b: dict, stream):
        mcdi.denoise_fwd(self.den_weights, b["terms"], b["kd_out"], b["gb"].nrm, b["den"], b["acts"], self.err, stream)
        mcdi.composite(b["kd_out"], b["den"][0:1], b["den"][1:2], b["color"], stream)

    def _capture_tails(self):
        """One CUDA graph per (side, slot) of the denoiser and the composite (launch
        parameters and tensor maps baked in for the slot's buffers at that size);
        a request replays it after its shading launches.  The convolutions are
        captured without their programmatic dependence: requests on the other
        slots run beside a replay, and a dependent launch's blocks would hold SM
        slots while they wait (measured at 400 requests/s: size-lane p50 3.33 ms
        without, 3.65 ms with)."""
        mcdi.set_graph_dependent_launch(False)
        try:
            self._capture_tail_graphs()
        finally:
            mcdi.set_graph_dependent_launch(True)

    def _capture_tail_graphs(self):
        for k, sl in enumerate(self.slots):
            s = self.streams[k]
            for r in self.sides:
                b = dict(sl.view(r), acts=sl.acts)
                with torch.cuda.stream(s):  # uncaptured once: one-time set-up stays outside the graph
                    self._tail(b, s)
                s.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.stream(s):
                    g.capture_begin()
                    self._tail(b, s)
                    g.capture_end()
                sl.graphs[r] = g
        torch.cuda.synchronize(self.dev)

    # ---- memory
    def footprint(self, req: RenderRequest) -> int:
        key = (req.res, req.spp)
        if key not in self._footprints:
            self._footprints[key] = self._footprint(req)
        return self._footprints[key]

    def _footprint(self, req: RenderRequest) -> int:
        P = req.res * req.res
        prm = mcdi.make_params(*split_spp(req.spp), seed=1)
        ws = mcdi.shade_workspace_size(1, req.res, req.res, prm)
        _, acts, _, _ = mcdi.denoise_sizes(2, req.res, req.res)
        rws = mcdi.raster_workspace_size(1, req.res, req.res)
        # G-buffer 4 planes, 2 terms, k_d out, 2 denoised, colour: float4 each
        return P * 16 * (4 + 2 + 1 + 2 + 1) + ws + acts + rws

    def _launch(self, req: RenderRequest, slot: int, stream):
        """The request on `stream`: camera into the slot, rasterised G-buffer and the shading
        forward (scene- and probe-dependent launches), then the slot's captured tail."""
        if req.res not in self.slots[slot].graphs or req.spp > self.max_spp:
            raise ValueError(f"request size {req.res} / {req.spp} spp outside the engine's sizes")
        sl, sc, pr = self.slots[slot], self.scenes[req.scene], self.probes[req.probe]
        b = sl.view(req.res)
        r = req.res
        sl.cam.copy_(sc.cams[req.view:req.view + 1], non_blocking=True)
        prm = mcdi.make_params(*split_spp(req.spp), seed=req.seed, tau=self.tau)
        mcdi.raster_gbuffer(sc.verts, sc.vnrm, sc.tris, sl.cam, r, r, sc.tex_kd, sc.tex_korm, sc.uvmap, b["gb"], sl.rws,
                            stream)
        mcdi.shade_mc_fwd(sc.bvh, pr, b["gb"], sl.cam, prm, b["terms"][0:1], b["kd_out"], b["terms"][1:2], None, sl.ws,
                          stream)
        sl.graphs[r].replay()
        return b

    def _lane_streams(self, n_lanes: int):
        """Streams for lanes 0..n_lanes-1 (lane i on slot i), lane n_lanes-1 (the largest
        requests) at the highest priority the device offers, the others at the lowest."""
        key = n_lanes
        if key not in self._lanes:
            lo, hi = torch.cuda.Stream.priority_range()
            self._lanes[key] = [torch.cuda.Stream(self.dev, priority=(hi if i == n_lanes - 1 else lo))
                                for i in range(n_lanes)]
        return self._lanes[key]

    def render_one(self, req: RenderRequest) -> np.ndarray:
        """Render a request alone (synchronously) and return its colour image."""
        s = self.streams[0]
        with torch.cuda.stream(s):
            b = self._launch(req, 0, s)
        s.synchronize()
        return b["color"][0].cpu().numpy()

    # ---- the loop
    def run(self, requests, mode: str = "continuous", keep=None, time_scale: float = 1.0, lanes=None):
        """Serve ``requests`` in real time (arrival times scaled by ``time_scale``).

        mode "continuous": requests are admitted while others are in flight.
        With ``lanes`` = (t_1, ..., t_{k-1}) sample-count bounds, a request of
        res^2 spp samples joins lane i, the first with samples < t_{i+1} (the
        last lane takes the rest); each lane serves its queue in arrival order
        on its own slot, lanes of larger requests on streams of higher priority,
        so that a small request does not wait behind a large one and a large one
        is slowed little by the small ones beside it.  Without ``lanes`` every
        slot serves the one queue in arrival order.  The HBM budget bounds the
        summed footprint of the requests in flight.  mode "serial": one request
        at a time in arrival order.  Returns a dict with per-request latency
        (ms, completion minus arrival), throughput and the colour images of the
        request ids in ``keep``."""
        if mode == "continuous" and lanes:
            bounds = list(lanes)
            n_lanes = len(bounds) + 1
            assert n_lanes <= self.n_slots
            # lane i runs on slot i; lanes of larger requests on the higher-priority streams
            lane_of = lambda q: sum(q.res * q.res * q.spp >= b for b in bounds)
            slot_of_lane = list(range(n_lanes))
            streams = self._lane_streams(n_lanes)
        else:
            n_lanes = 1
            lane_of = lambda q: 0
            slot_of_lane = None
            streams = self.streams[: (self.n_slots if mode == "continuous" else 1)]
        keep = set(keep or ())
        reqs = sorted(requests, key=lambda q: q.arrival)
        pending = [deque() for _ in range(n_lanes)]
        free = list(range(len(streams))) if slot_of_lane is None else None
        busy = [False] * n_lanes
        inflight = {}
        used = 0
        lat = np.zeros(len(reqs))
        images = {}
        nxt = 0
        n_done = 0
        refused = 0
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        while n_done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival * time_scale <= now:
                pending[lane_of(reqs[nxt])].append(reqs[nxt])
                nxt += 1
            # completions
            for slot, fl in list(inflight.items()):
                if fl.event.query():
                    tdone = time.perf_counter() - t0
                    i = fl.req.rid
                    lat[i] = (tdone - fl.req.arrival * time_scale) * 1e3
                    if i in keep:
                        images[i] = self.slots[slot].view(fl.req.res)["color"][0].cpu().numpy()
                    used -= fl.bytes
                    del inflight[slot]
                    if free is not None:
                        free.append(slot)
                    else:
                        busy[slot_of_lane.index(slot)] = False
                    n_done += 1
            # admission: per lane in arrival order while a slot is free and the footprint fits
            for ln in range(n_lanes):
                q = pending[ln]
                while q and (free if free is not None else not busy[ln]):
                    req = q[0]
                    need = self.footprint(req)
                    if used + need > self.hbm_budget and inflight:
                        refused += 1
                        break
                    q.popleft()
                    if free is not None:
                        slot = free.pop(0)
                        s = streams[slot]
                    else:
                        slot = slot_of_lane[ln]
                        s = streams[ln]
                        busy[ln] = True
                    with torch.cuda.stream(s):
                        self._launch(req, slot, s)
                        ev = torch.cuda.Event()
                        ev.record(s)
                    inflight[slot] = _InFlight(req, ev, need, slot)
                    used += need
            if not inflight and nxt < len(reqs) and not any(pending):
                # idle until the next arrival: sleep while it is more than a millisecond
                # away, then poll, so that an arrival is seen within microseconds
                wait = reqs[nxt].arrival * time_scale - (time.perf_counter() - t0)
                if wait > 1e-3:
                    time.sleep(min(wait - 5e-4, 2e-3))
        total = time.perf_counter() - t0
        if self.err.item() != 0:
            raise RuntimeError("a denoiser pipeline wait timed out")
        samples = sum(q.res * q.res * q.spp for q in reqs)
        return {"mode": mode, "n": len(reqs), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "wall_s": total,
                "req_per_s": len(reqs) / total, "msamples_per_s": samples / total / 1e6, "admission_waits": refused,
                "latency_ms": lat, "images": images}
