"""Serving (continuous batching in one persistent kernel): each request's result
is the same alone and in a mix, hard requests equal the plain entry point bit
for bit and soft requests match it to FP32 rounding (the serving kernel runs the
soft forward two pixels per thread from a per-CTA record, the plain path one
pixel per thread), edits render the edited program, admission respects the
memory cap, and the kernel is relaunched after it exits idle."""
import time

import numpy as np
import pytest
import torch

from paper_2609_08722_b300 import inputs, tbr

pytestmark = pytest.mark.gpu

GROUPS = ["cx", "cy", "theta", "length", "half_width", "logits"]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def server():
    s = tbr.Server(tbr.default_serve_config(max_strokes=4096))
    yield s
    s.destroy()


@pytest.fixture(scope="module")
def programs():
    hs = [inputs.make_program(n, seed=3000 + j, palette_seed=77, k=16, r_lo=0.003, r_hi=0.05)
          for j, n in enumerate((200, 700, 2000))]
    return hs, [tbr.DeviceProgram.from_host(h) for h in hs]


class MappedWord:
    """One int32 in mapped pinned host memory (cudaHostAllocMapped): the host
    writes it, kernels read it through its device address."""

    def __init__(self):
        from cuda.bindings import runtime as rt
        self.rt = rt
        err, self.host = rt.cudaHostAlloc(4, rt.cudaHostAllocMapped)
        assert err == rt.cudaError_t.cudaSuccess
        err, self.dev = rt.cudaHostGetDevicePointer(self.host, 0)
        assert err == rt.cudaError_t.cudaSuccess
        self.set(0)

    def set(self, v):
        import ctypes
        ctypes.c_int32.from_address(int(self.host)).value = v

    def device_view(self):
        class _View:  # what Server.submit needs of a ready tensor
            dtype = torch.int32

            def __init__(self, ptr):
                self._p = ptr

            def data_ptr(self):
                return self._p
        return _View(int(self.dev))

    def free(self):
        self.rt.cudaFreeHost(self.host)


def hard_request(server, pid, W, H):
    rgb = torch.full((H, W, 3), float("nan"), device="cuda")
    idx = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
    rid = server.submit(tbr.REQ_HARD, pid, W, H, out_rgb=rgb, out_idx=idx)
    return rid, rgb, idx


def soft_request(server, pid, n, k, target, tau=0.0, tau_min=1 / 200):
    H, W = target.shape[0], target.shape[1]
    grad = torch.full((5 * n + n * k,), float("nan"), device="cuda")
    loss = torch.full((1,), float("nan"), device="cuda")
    rgb = torch.empty((H, W, 3), device="cuda")
    rid = server.submit(tbr.REQ_SOFT_ADJOINT, pid, W, H, out_rgb=rgb, target=target, out_loss=loss,
                        out_grad=grad, tau=tau, tau_min=tau_min)
    return rid, rgb, loss, grad


def split_grad(g, n, k):
    return {"cx": g[:n], "cy": g[n:2 * n], "theta": g[2 * n:3 * n], "length": g[3 * n:4 * n],
            "half_width": g[4 * n:5 * n], "logits": g[5 * n:].view(n, k)}


def test_hard_request_equals_plain_hard_render(server, programs):
    hs, ds = programs
    for dp, (W, H) in zip(ds, [(256, 256), (333, 97), (512, 512)]):
        pid = server.load_program(dp)
        rid, rgb, idx = hard_request(server, pid, W, H)
        assert server.wait(rid) == tbr.TBR_OK
        ref_rgb, ref_idx, _ = tbr.render_hard(dp, W, H)
        torch.cuda.synchronize()
        assert torch.equal(idx, ref_idx)
        assert torch.equal(rgb, ref_rgb)


def test_soft_request_matches_the_fused_entry_point(server, programs):
    hs, ds = programs
    dp = ds[1]
    W, H = 192, 160
    target, _, _ = tbr.render_hard(ds[0], W, H)
    pid = server.load_program(dp)
    rid, rgb, loss, grad = soft_request(server, pid, dp.n, dp.k, target)
    assert server.wait(rid) == tbr.TBR_OK
    loss_f, g_f, rgb_f, _ = tbr.soft_adjoint_mse(dp, target, 0.0, 1 / 200, want_rgb=True)
    torch.cuda.synchronize()
    assert (rgb - rgb_f).abs().max().item() <= 1e-5
    assert abs(loss.item() - loss_f.item()) <= 1e-5 * abs(loss_f.item())
    g = split_grad(grad, dp.n, dp.k)
    for k in GROUPS:
        assert rel(g[k].cpu().numpy().ravel(), g_f[k].cpu().numpy().ravel()) <= 1e-4, k


def test_results_are_identical_alone_and_in_a_mix(server, programs):
    hs, ds = programs
    pids = [server.load_program(d) for d in ds]
    W, H = 160, 128
    target, _, _ = tbr.render_hard(ds[2], W, H)
    # alone
    alone = []
    for j, (pid, d) in enumerate(zip(pids, ds)):
        rid, rgb, idx = hard_request(server, pid, W + 32 * j, H)
        server.wait(rid)
        rs, srgb, sloss, sgrad = soft_request(server, pid, d.n, d.k, target)
        server.wait(rs)
        alone.append((rgb.clone(), idx.clone(), sloss.clone(), sgrad.clone()))
    # mixed: everything submitted at once, interleaved kinds
    mixed = []
    rids = []
    for j, (pid, d) in enumerate(zip(pids, ds)):
        rid, rgb, idx = hard_request(server, pid, W + 32 * j, H)
        rs, srgb, sloss, sgrad = soft_request(server, pid, d.n, d.k, target)
        rids += [rid, rs]
        mixed.append((rgb, idx, sloss, sgrad))
    for rid in rids:
        assert server.wait(rid) == tbr.TBR_OK
    torch.cuda.synchronize()
    for a, m in zip(alone, mixed):
        for x, y in zip(a, m):
            assert torch.equal(x, y)


@pytest.mark.parametrize("kind", [tbr.REQ_RECOLOUR, tbr.REQ_REORDER, tbr.REQ_INSERT])
def test_edit_requests_render_the_edited_program(server, programs, kind):
    hs, ds = programs
    h = hs[1]
    pid = server.load_program(ds[1])
    W, H = 200, 150
    n = h.n
    e = h.copy()
    args = {}
    if kind == tbr.REQ_RECOLOUR:
        a, b, start = 2, 9, 4 * n // 5
        lg = e.logits.copy()
        lg[start:, [a, b]] = lg[start:, [b, a]]
        e.logits = np.ascontiguousarray(lg)
        args = dict(edit_a=a, edit_b=b, edit_start=start)
    elif kind == tbr.REQ_REORDER:
        start, length = 300, 16
        for name in ("cx", "cy", "theta", "length", "half_width", "logits"):
            arr = getattr(e, name).copy()
            arr[start:start + length] = arr[start:start + length][::-1]
            setattr(e, name, np.ascontiguousarray(arr))
        args = dict(edit_b=length, edit_start=start)
    else:
        at, stroke, pal = n // 2, (0.45, 0.55, 0.0, 0.0, 0.06), 5
        for name, v in zip(("cx", "cy", "theta", "length", "half_width"), stroke):
            setattr(e, name, np.ascontiguousarray(np.insert(getattr(e, name), at, np.float32(v))))
        z = np.zeros((1, h.k), np.float32)
        z[0, pal] = 6.0
        e.logits = np.ascontiguousarray(np.insert(e.logits, at, z, axis=0))
        args = dict(edit_start=at, insert_palette=pal, insert_stroke=stroke)
    rgb = torch.empty((H, W, 3), device="cuda")
    idx = torch.empty((H, W), dtype=torch.int32, device="cuda")
    rid = server.submit(kind, pid, W, H, out_rgb=rgb, out_idx=idx, **args)
    assert server.wait(rid) == tbr.TBR_OK
    ref_rgb, ref_idx, _ = tbr.render_hard(tbr.DeviceProgram.from_host(e), W, H)
    torch.cuda.synchronize()
    assert torch.equal(idx, ref_idx)
    assert torch.equal(rgb, ref_rgb)
    if kind == tbr.REQ_RECOLOUR:
        # transport ignores pigment: the index map of a recolour edit is the original one
        _, idx0, _ = tbr.render_hard(ds[1], W, H)
        assert torch.equal(idx, idx0)


def test_admission_respects_the_memory_cap(programs):
    hs, ds = programs
    s = tbr.Server(tbr.default_serve_config(memory_cap_bytes=1 << 20, max_strokes=4096))
    try:
        pid = s.load_program(ds[2])
        W, H = 128, 128
        target, _, _ = tbr.render_hard(ds[0], W, H)
        with pytest.raises(tbr.TbrError) as ei:      # a 2000-stroke soft request never fits 1 MiB
            soft_request(s, pid, ds[2].n, ds[2].k, target)
        assert ei.value.status == tbr.TBR_ERR_ADMISSION
        outs = [hard_request(s, pid, W, H) for _ in range(6)]   # ~260 KB each: at most a few at a time
        for rid, _, _ in outs:
            assert s.wait(rid) == tbr.TBR_OK
        ref_rgb, ref_idx, _ = tbr.render_hard(ds[2], W, H)
        torch.cuda.synchronize()
        for _, rgb, idx in outs:
            assert torch.equal(idx, ref_idx)
        st = s.stats()
        assert st["completed"] == 6 and st["bytes_in_use"] == 0
    finally:
        s.destroy()


def test_kernel_relaunches_after_idle(server, programs):
    hs, ds = programs
    pid = server.load_program(ds[0])
    before = server.stats()["kernel_launches"]
    rid, _, _ = hard_request(server, pid, 64, 64)
    assert server.wait(rid) == tbr.TBR_OK
    time.sleep(0.05)  # > idle_exit_us: the persistent kernel has exited
    rid, rgb, idx = hard_request(server, pid, 64, 64)
    assert server.wait(rid) == tbr.TBR_OK
    assert server.stats()["kernel_launches"] >= before + 1
    ref_rgb, ref_idx, _ = tbr.render_hard(ds[0], 64, 64)
    torch.cuda.synchronize()
    assert torch.equal(idx, ref_idx)


def test_ready_word_wait_runs_out_and_the_server_stays_usable(programs):
    """A request whose ready word is never set: every item's bounded device wait
    gives up after ready_wait_us, the request completes with TBR_ERR_TIMEOUT and
    leaves its outputs untouched, and the server goes on serving: a request
    whose word is set later (before the limit) and one without a word render
    the plain path's result.  No GPU fault or trap is involved: the wait is a
    polled loop on the device clock that returns a status."""
    hs, dps = programs
    s = tbr.Server(tbr.default_serve_config(max_strokes=4096, ready_wait_us=3000))
    try:
        pid = s.load_program(dps[1])
        W, H = 96, 64
        never = torch.zeros(1, dtype=torch.int32, device="cuda")
        rgb0 = torch.full((H, W, 3), float("nan"), device="cuda")
        idx0 = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        r0 = s.submit(tbr.REQ_HARD, pid, W, H, out_rgb=rgb0, out_idx=idx0, ready=never)
        assert s.wait(r0) == tbr.TBR_ERR_TIMEOUT
        assert torch.isnan(rgb0).all() and (idx0 == -7).all()
        t = torch.full((H, W, 3), 0.5, device="cuda")
        r0s = s.submit(tbr.REQ_SOFT_ADJOINT, pid, W, H, target=t, out_loss=torch.zeros(1, device="cuda"),
                       out_grad=torch.zeros(5 * hs[1].n + hs[1].n * hs[1].k, device="cuda"), ready=never)
        assert s.wait(r0s) == tbr.TBR_ERR_TIMEOUT
        # set later by a host thread writing mapped pinned memory while the
        # request waits (limit raised for it): the producer outside stream order
        s2 = tbr.Server(tbr.default_serve_config(max_strokes=4096, ready_wait_us=2000000))
        word = MappedWord()
        try:
            pid2 = s2.load_program(dps[1])
            rgb = torch.full((H, W, 3), float("nan"), device="cuda")
            idx = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            rid = s2.submit(tbr.REQ_HARD, pid2, W, H, out_rgb=rgb, out_idx=idx, ready=word.device_view())
            time.sleep(0.05)
            word.set(1)
            assert s2.wait(rid) == tbr.TBR_OK
            ref_rgb, ref_idx, _ = tbr.render_hard(dps[1], W, H)
            assert torch.equal(idx, ref_idx) and torch.equal(rgb, ref_rgb)
        finally:
            s2.destroy()
            word.free()
        # the first server still serves
        rid, rgb, idx = hard_request(s, pid, W, H)
        assert s.wait(rid) == tbr.TBR_OK
        ref_rgb, ref_idx, _ = tbr.render_hard(dps[1], W, H)
        assert torch.equal(idx, ref_idx) and torch.equal(rgb, ref_rgb)
    finally:
        s.destroy()


def test_random_mix_matches_alone_and_the_plain_path():
    """80 random requests over 12 random programs (1 .. 4000 strokes; 1 .. 333
    pixels a side), submitted at once: hard and recolour requests equal the
    plain entry point bit for bit, and every soft request, resubmitted alone,
    reproduces its in-mix colours, loss and gradients bit for bit (the mix
    never reorders a request's own arithmetic)."""
    rng = np.random.default_rng(5)
    s = tbr.Server(tbr.default_serve_config(max_strokes=4096))
    try:
        hosts, devs, pids = [], [], []
        for j in range(12):
            n = int(rng.choice([1, 50, 300, 1000, 4000]))
            r_lo = float(rng.choice([0.003, 0.01]))
            h = inputs.make_program(n, seed=7600 + j, palette_seed=78, k=int(rng.choice([4, 16])), r_lo=r_lo,
                                    r_hi=r_lo * 8)
            d = tbr.DeviceProgram.from_host(h)
            hosts.append(h)
            devs.append(d)
            pids.append(s.load_program(d))
        reqs = []
        for _ in range(80):
            j = int(rng.integers(0, 12))
            W, H = int(rng.choice([1, 17, 64, 130, 256, 333])), int(rng.choice([1, 9, 64, 100, 256]))
            u = rng.random()
            if u < 0.6:
                rid, rgb, idx = hard_request(s, pids[j], W, H)
                reqs.append(("hard", j, W, H, rid, (rgb, idx)))
            elif u < 0.9:
                target, _, _ = tbr.render_hard(devs[(j + 1) % 12], W, H)
                rid, rgb, loss, grad = soft_request(s, pids[j], devs[j].n, devs[j].k, target)
                reqs.append(("soft", j, W, H, rid, (rgb, loss, grad, target)))
            else:
                a, b, start = 0, hosts[j].k - 1, hosts[j].n // 2
                rgb = torch.empty((H, W, 3), device="cuda")
                idx = torch.empty((H, W), dtype=torch.int32, device="cuda")
                rid = s.submit(tbr.REQ_RECOLOUR, pids[j], W, H, out_rgb=rgb, out_idx=idx, edit_a=a, edit_b=b,
                               edit_start=start)
                reqs.append(("recolour", j, W, H, rid, (rgb, idx, a, b, start)))
        for kind, j, W, H, rid, out in reqs:
            assert s.wait(rid) == tbr.TBR_OK
        torch.cuda.synchronize()
        for kind, j, W, H, rid, out in reqs:
            if kind == "hard":
                ref_rgb, ref_idx, _ = tbr.render_hard(devs[j], W, H)
                assert torch.equal(out[1], ref_idx) and torch.equal(out[0], ref_rgb), (kind, j, W, H)
            elif kind == "recolour":
                rgb, idx, a, b, start = out
                e = hosts[j].copy()
                lg = e.logits.copy()
                lg[start:, [a, b]] = lg[start:, [b, a]]
                e.logits = np.ascontiguousarray(lg)
                ref_rgb, ref_idx, _ = tbr.render_hard(tbr.DeviceProgram.from_host(e), W, H)
                assert torch.equal(idx, ref_idx) and torch.equal(rgb, ref_rgb), (kind, j, W, H)
            else:
                rgb, loss, grad, target = out
                rid2, rgb2, loss2, grad2 = soft_request(s, pids[j], devs[j].n, devs[j].k, target)
                assert s.wait(rid2) == tbr.TBR_OK
                torch.cuda.synchronize()
                assert torch.equal(rgb, rgb2) and torch.equal(loss, loss2) and torch.equal(grad, grad2), (kind, j, W, H)
    finally:
        s.destroy()
