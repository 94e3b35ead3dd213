"""Serving benchmark: a seeded Poisson stream of mixed requests against the
continuous-batching server, and the same stream through one-program-per-launch
replay (each request is one plain C-ABI call, run in arrival order on one
stream), both reporting p50 / p99 latency (arrival to completion) and
throughput.

Request mix (the serving workload): 60% hard re-render, 30% soft render +
replay adjoint against a target, 10% edit (recolour: swap two palette entries
over the last fifth of the strokes; reorder: reverse a window of 16 strokes;
insert: a drop of r = 0.06 at the middle index); programs of 200-5000 strokes
(log-uniform) resident on the device; resolutions 256^2, 512^2, 1024^2 or
2048^2 (uniform); admission under an 80 GB device-memory cap.
"""
from __future__ import annotations

import math
import sys
import time

import numpy as np
import torch

from . import inputs, tbr

RESOLUTIONS = (256, 512, 1024, 2048)


def make_stream(n_req: int, n_prog: int, seed: int):
    u = inputs.uniform(seed, 6 * n_req).reshape(n_req, 6)
    reqs = []
    for j in range(n_req):
        kind_u = u[j, 0]
        if kind_u < 0.6:
            kind = tbr.REQ_HARD
        elif kind_u < 0.9:
            kind = tbr.REQ_SOFT_ADJOINT
        else:
            kind = (tbr.REQ_RECOLOUR, tbr.REQ_REORDER, tbr.REQ_INSERT)[min(2, int(u[j, 1] * 3))]
        prog = min(n_prog - 1, int(u[j, 2] * n_prog))
        res = RESOLUTIONS[min(3, int(u[j, 3] * 4))]
        reqs.append({"kind": kind, "prog": prog, "res": res, "u": float(u[j, 4])})
    return reqs


def make_programs(n_prog: int, seed: int):
    """n_prog seeded programs, stroke counts log-uniform in [200, 5000]."""
    u = inputs.uniform(seed, n_prog)
    out = []
    for j in range(n_prog):
        n = int(round(math.exp(math.log(200) + u[j] * (math.log(5000) - math.log(200)))))
        out.append(inputs.make_program(n, seed=1000 + j, palette_seed=501, k=16, r_lo=0.003, r_hi=0.05))
    return out


def _edit_args(req, n):
    if req["kind"] == tbr.REQ_RECOLOUR:
        return dict(edit_a=1, edit_b=2, edit_start=(4 * n) // 5)
    if req["kind"] == tbr.REQ_REORDER:
        start = min(max(0, int(req["u"] * (n - 16))), max(0, n - 16))
        return dict(edit_b=min(16, n), edit_start=start)
    if req["kind"] == tbr.REQ_INSERT:
        return dict(edit_start=n // 2, insert_palette=3, insert_stroke=(0.5, 0.5, 0.0, 0.0, 0.06))
    return {}


def _host_edit(prog, req):
    """The edited program on the host (for the one-program-per-launch arm)."""
    e = prog.copy()
    n = prog.n
    a = _edit_args(req, n)
    if req["kind"] == tbr.REQ_RECOLOUR:
        lg = e.logits.copy()
        s = a["edit_start"]
        lg[s:, [a["edit_a"], a["edit_b"]]] = lg[s:, [a["edit_b"], a["edit_a"]]]
        e.logits = np.ascontiguousarray(lg)
    elif req["kind"] == tbr.REQ_REORDER:
        s, L = a["edit_start"], a["edit_b"]
        for name in ("cx", "cy", "theta", "length", "half_width", "logits"):
            arr = getattr(e, name).copy()
            arr[s:s + L] = arr[s:s + L][::-1]
            setattr(e, name, np.ascontiguousarray(arr))
    elif req["kind"] == tbr.REQ_INSERT:
        at = a["edit_start"]
        for name, v in zip(("cx", "cy", "theta", "length", "half_width"), a["insert_stroke"]):
            setattr(e, name, np.ascontiguousarray(np.insert(getattr(e, name), at, np.float32(v))))
        z = np.zeros((1, prog.k), np.float32)
        z[0, a["insert_palette"]] = 6.0
        e.logits = np.ascontiguousarray(np.insert(e.logits, at, z, axis=0))
    return e


def _percentiles(lat):
    a = np.sort(np.asarray(lat))
    return float(np.percentile(a, 50)), float(np.percentile(a, 99)), float(a.mean())


class _Bench:
    def __init__(self, n_prog, seed):
        self.hosts = make_programs(n_prog, seed)
        self.devs = [tbr.DeviceProgram.from_host(h) for h in self.hosts]
        self.targets = {r: tbr.render_hard(self.devs[0], r, r, with_idx=False)[0] for r in RESOLUTIONS}
        self.edited = {}

    def outputs(self, req):
        r = req["res"]
        d = self.devs[req["prog"]]
        if req["kind"] == tbr.REQ_SOFT_ADJOINT:
            n, k = d.n, d.k
            return {"out_grad": torch.empty(5 * n + n * k, device="cuda"),
                    "out_loss": torch.empty(1, device="cuda"), "target": self.targets[r]}
        return {"out_rgb": torch.empty((r, r, 3), device="cuda"),
                "out_idx": torch.empty((r, r), dtype=torch.int32, device="cuda")}

    # -- continuous batching ------------------------------------------------------
    def run_server(self, stream, arrivals, server, pids):
        self.queue_ms = []
        lat = [None] * len(stream)
        rids = [None] * len(stream)
        t0 = time.perf_counter()
        keep = []
        for j, (req, ta) in enumerate(zip(stream, arrivals)):
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            o = self.outputs(req)
            keep.append(o)
            d = self.devs[req["prog"]]
            kw = dict(o)
            if req["kind"] == tbr.REQ_SOFT_ADJOINT:
                kw.update(tau=0.0, tau_min=1 / 200)
            kw.update(_edit_args(req, d.n))
            rids[j] = server.submit(req["kind"], pids[req["prog"]], req["res"], req["res"], **kw)
        for j, rid in enumerate(rids):
            try:
                server.wait(rid, 120000)
            except tbr.TbrError:
                print(f"serve_bench: request {j} ({stream[j]}) not done; server {server.stats()}",
                      file=sys.stderr, flush=True)
                raise
            qms, lms = server.times(rid)
            lat[j] = lms
            self.queue_ms.append(qms)
            server.release(rid)
        wall = time.perf_counter() - t0
        return lat, wall

    # -- one program per launch -------------------------------------------------
    def run_per_launch(self, stream, arrivals):
        lat = []
        t0 = time.perf_counter()
        for req, ta in zip(stream, arrivals):
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            r = req["res"]
            if req["kind"] == tbr.REQ_SOFT_ADJOINT:
                tbr.soft_adjoint_mse(self.devs[req["prog"]], self.targets[r], 0.0, 1 / 200)
            else:
                d = self.devs[req["prog"]]
                if req["kind"] != tbr.REQ_HARD:
                    key = (req["prog"], req["kind"], int(req["u"] * 1e6))
                    d = tbr.DeviceProgram.from_host(_host_edit(self.hosts[req["prog"]], req))
                tbr.render_hard(d, r, r)
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - t0 - ta) * 1e3)
        return lat, time.perf_counter() - t0


def run(n_req: int = 200, n_prog: int = 64, rho: float = 0.7, seed: int = 501, cap_bytes: int = 80 << 30,
        sweep=(0.3, 0.5, 0.9, 1.2)):
    """Returns a dict with capacity, and p50/p99 latency of both arms at
    ``rho`` x the server's measured capacity; ``rate_sweep`` repeats the
    Poisson run of both arms at each further load in ``sweep`` (the same
    seeded draws, gaps scaled by 1 / load)."""
    b = _Bench(n_prog, seed)
    stream = make_stream(n_req, n_prog, seed + 1)
    server = tbr.Server(tbr.default_serve_config(memory_cap_bytes=cap_bytes, max_strokes=8192))
    try:
        pids = [server.load_program(d) for d in b.devs]
        # warm-up and capacity: the whole stream submitted at once
        t0 = time.perf_counter()
        warm = make_stream(20, n_prog, seed + 7)
        b.run_server(warm, [0.0] * len(warm), server, pids)
        print(f"serve_bench: warm-up {time.perf_counter() - t0:.1f} s", file=sys.stderr, flush=True)
        lat_cap, wall_cap = b.run_server(stream, [0.0] * len(stream), server, pids)
        print(f"serve_bench: capacity run {wall_cap:.1f} s", file=sys.stderr, flush=True)
        capacity = len(stream) / wall_cap
        # Poisson arrivals at rho x capacity
        unit = -np.log(1.0 - inputs.uniform(seed + 2, len(stream))) / capacity

        def schedule(load):
            gaps = unit / load
            return (np.cumsum(gaps) - gaps[0]).tolist()

        arrivals = schedule(rho)
        lat_s, wall_s = b.run_server(stream, arrivals, server, pids)
        queue_s = float(np.mean(b.queue_ms))
        st = server.stats()
        swept = {}
        for load in sweep:
            lat, wall = b.run_server(stream, schedule(load), server, pids)
            swept[load] = {"server": _arm(lat, wall, len(stream))}
    finally:
        server.destroy()
    print(f"serve_bench: poisson run {wall_s:.1f} s", file=sys.stderr, flush=True)
    b.run_per_launch(make_stream(10, n_prog, seed + 7), [0.0] * 10)
    lat_p, wall_p = b.run_per_launch(stream, arrivals)
    for load in sweep:
        lat, wall = b.run_per_launch(stream, schedule(load))
        swept[load]["per_launch"] = _arm(lat, wall, len(stream))
    print(f"serve_bench: per-launch poisson run {wall_p:.1f} s", file=sys.stderr, flush=True)
    lat_pc, wall_pc = b.run_per_launch(stream, [0.0] * len(stream))
    p50s, p99s, means = _percentiles(lat_s)
    p50p, p99p, meanp = _percentiles(lat_p)
    return {
        "requests": len(stream), "programs": n_prog, "arrival_rate_per_s": rho * capacity, "rho": rho,
        "mix": "60% hard, 30% soft+adjoint, 10% edit; 200-5000 strokes; 256^2-2048^2",
        "server": {"capacity_req_per_s": capacity, "p50_ms": p50s, "p99_ms": p99s, "mean_ms": means,
                   "mean_admission_wait_ms": queue_s,
                   "throughput_req_per_s": len(stream) / wall_s, "kernel_launches": st["kernel_launches"],
                   "persistent_ctas": st["persistent_ctas"]},
        "per_launch": {"capacity_req_per_s": len(stream) / wall_pc, "p50_ms": p50p, "p99_ms": p99p,
                       "mean_ms": meanp, "throughput_req_per_s": len(stream) / wall_p},
        "rate_sweep": [{"rho": load, "arrival_rate_per_s": load * capacity, **swept[load]} for load in sweep],
    }


def _arm(lat, wall, count):
    p50, p99, mean = _percentiles(lat)
    return {"p50_ms": p50, "p99_ms": p99, "mean_ms": mean, "throughput_req_per_s": count / wall}


if __name__ == "__main__":
    import json
    import sys
    print(json.dumps(run(n_req=int(sys.argv[1]) if len(sys.argv) > 1 else 200)))
