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
    bufs: dict = field(default_factory=dict)


class ServingEngine:
    def __init__(self, scene_list, probe_list, denoiser_params, n_slots: int = 4, hbm_budget: int = 8 << 30,
                 device="cuda", tau: float = 1.0):
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
        self.streams = [torch.cuda.Stream(dev) for _ in range(n_slots)]
        torch.cuda.synchronize(dev)

    # ---- memory
    def footprint(self, req: RenderRequest) -> int:
        P = req.res * req.res
        prm = mcdi.make_params(*split_spp(req.spp), seed=1)
        ws = mcdi.shade_workspace_size(1, req.res, req.res, prm)
        _, acts, _, _ = mcdi.denoise_sizes(2, req.res, req.res)
        rws = mcdi.raster_workspace_size(1, req.res, req.res)
        # G-buffer 4 planes, 2 terms, k_d out, 2 denoised, colour: float4 each
        return P * 16 * (4 + 2 + 1 + 2 + 1) + ws + acts + rws

    def _alloc(self, req: RenderRequest):
        dev, r = self.dev, req.res
        f4 = lambda n: torch.empty((n, r, r, 4), device=dev)
        prm = mcdi.make_params(*split_spp(req.spp), seed=req.seed, tau=self.tau)
        ws = mcdi.shade_workspace_size(1, r, r, prm)
        _, acts, _, _ = mcdi.denoise_sizes(2, r, r)
        gb = mcdi.GBuffer(f4(1), f4(1), f4(1), f4(1))
        rws = mcdi.raster_workspace_size(1, r, r)
        return dict(prm=prm, gb=gb, terms=f4(2), kd_out=f4(1), den=f4(2), color=f4(1),
                    ws=torch.empty((ws + 255) // 256 * 256, dtype=torch.uint8, device=dev),
                    rws=torch.empty((rws + 255) // 256 * 256, dtype=torch.uint8, device=dev),
                    acts=torch.empty((acts + 255) // 256 * 256, dtype=torch.uint8, device=dev))

    def _launch(self, req: RenderRequest, b: dict, stream):
        sc, pr = self.scenes[req.scene], self.probes[req.probe]
        cams = sc.cams[req.view:req.view + 1]
        r = req.res
        mcdi.raster_gbuffer(sc.verts, sc.vnrm, sc.tris, cams, r, r, sc.tex_kd, sc.tex_korm, sc.uvmap, b["gb"], b["rws"],
                            stream)
        c_d, c_s = b["terms"][0:1], b["terms"][1:2]
        mcdi.shade_mc_fwd(sc.bvh, pr, b["gb"], cams, b["prm"], c_d, b["kd_out"], c_s, None, b["ws"], stream)
        mcdi.denoise_fwd(self.den_weights, b["terms"], b["kd_out"], b["gb"].nrm, b["den"], b["acts"], self.err, stream)
        mcdi.composite(b["kd_out"], b["den"][0:1], b["den"][1:2], b["color"], stream)

    def render_one(self, req: RenderRequest) -> np.ndarray:
        """Render a request alone (synchronously) and return its colour image."""
        s = self.streams[0]
        with torch.cuda.stream(s):
            b = self._alloc(req)
            self._launch(req, b, s)
        s.synchronize()
        return b["color"][0].cpu().numpy()

    # ---- the loop
    def run(self, requests, mode: str = "continuous", keep=None, time_scale: float = 1.0):
        """Serve ``requests`` in real time (arrival times scaled by ``time_scale``).

        mode "continuous": up to n_slots requests in flight, admitted FIFO while
        the HBM budget allows; "serial": one at a time.  Returns a dict with
        per-request latency (ms, completion minus arrival), throughput and the
        colour images of the request ids in ``keep``."""
        n_slots = self.n_slots if mode == "continuous" else 1
        keep = set(keep or ())
        reqs = sorted(requests, key=lambda q: q.arrival)
        pending = deque()
        free = list(range(n_slots))
        inflight = {}
        used = 0
        lat = np.zeros(len(reqs))
        done_at = np.zeros(len(reqs))
        images = {}
        nxt = 0
        n_done = 0
        refused = 0
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        while n_done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival * time_scale <= now:
                pending.append(reqs[nxt])
                nxt += 1
            # completions
            for slot, fl in list(inflight.items()):
                if fl.event.query():
                    tdone = time.perf_counter() - t0
                    i = fl.req.rid
                    lat[i] = (tdone - fl.req.arrival * time_scale) * 1e3
                    done_at[i] = tdone
                    if i in keep:
                        images[i] = fl.bufs["color"][0].cpu().numpy()
                    used -= fl.bytes
                    del inflight[slot]
                    free.append(slot)
                    n_done += 1
            # admission: FIFO while a slot is free and the footprint fits
            while pending and free:
                req = pending[0]
                need = self.footprint(req)
                if used + need > self.hbm_budget and inflight:
                    refused += 1
                    break
                pending.popleft()
                slot = free.pop(0)
                s = self.streams[slot]
                with torch.cuda.stream(s):
                    bufs = self._alloc(req)
                    self._launch(req, bufs, s)
                    ev = torch.cuda.Event()
                    ev.record(s)
                inflight[slot] = _InFlight(req, ev, need, bufs)
                used += need
            if not inflight and nxt < len(reqs) and not pending:
                # idle until the next arrival
                wait = reqs[nxt].arrival * time_scale - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
        total = time.perf_counter() - t0
        if self.err.item() != 0:
            raise RuntimeError("a denoiser pipeline wait timed out")
        samples = sum(q.res * q.res * q.spp for q in reqs)
        return {"mode": mode, "n": len(reqs), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "wall_s": total,
                "req_per_s": len(reqs) / total, "msamples_per_s": samples / total / 1e6, "admission_waits": refused,
                "latency_ms": lat, "images": images}
