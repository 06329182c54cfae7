"""GPU tests of the continuous-batching server (fcfs_serve_*).

Results must not depend on the mix: every request's output is compared with
the same request run alone, and with the standalone forward, bit for bit; a
few are also checked against the FP64 oracle.  Admission under a tiny pool,
timeouts, rejections and malformed requests are exercised on the host side
(no GPU fault is induced)."""
import math

import numpy as np
import pytest
import torch

from paper_2203_10670_gb300 import inputs

pytestmark = pytest.mark.gpu

RATIOS = inputs.C4["ratios"]


@pytest.fixture(scope="module")
def F():
    from paper_2203_10670_gb300 import build

    build.build()
    from paper_2203_10670_gb300 import fcfs

    return fcfs


def _requests(count, seed, lo=16, hi=300):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        H = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        W = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        r, s = RATIOS[rng.integers(0, len(RATIOS))]
        m = int(rng.integers(0, 3))
        x = inputs.uint8_pixels((1, 3, H, W), 1000 + seed * 10000 + k, device="cuda")
        out.append((x, (r, s), m))
    return out


def _run(F, reqs, out_dtype, **cfg):
    outs = []
    with F.Server(1 << 30, out_dtype=out_dtype, **cfg) as sv:
        ids = []
        for x, ratio, m in reqs:
            y = torch.empty(F.out_shape(x.shape, [F.Axis(*ratio, m)] * 2), device="cuda", dtype=out_dtype)
            ids.append(sv.submit(x, ratio, m, y=y))
            outs.append(y)
        sv.drain(60_000)
        done = set()
        while len(done) < len(ids):
            got = sv.poll()
            assert got or len(done) == len(ids)
            done.update(got)
        assert done == set(ids)
        st = sv.stats()
    torch.cuda.synchronize()
    return outs, st


@pytest.mark.parametrize("out_dtype", (torch.float32, torch.bfloat16))
def test_mixed_equals_alone_and_standalone(F, orc, out_dtype):
    reqs = _requests(120, 1)
    mixed, st = _run(F, reqs, out_dtype, max_inflight=32, tile_budget_per_step=64)
    assert st["completed"] == len(reqs) and st["steps"] > 1 and st["max_inflight_seen"] > 1
    assert st["p50_ms"] <= st["p99_ms"]
    alone, _ = _run(F, reqs, out_dtype, max_inflight=1, tile_budget_per_step=4096)
    for (x, ratio, m), a, b in zip(reqs, mixed, alone):
        assert torch.equal(a, b)  # independent of the mix
        ref = F.resize(x, [F.Axis(*ratio, m)] * 2, out_dtype=out_dtype)
        assert torch.equal(a, ref)  # and of the launch path
    for (x, ratio, m), a in list(zip(reqs, mixed))[:12]:
        want = orc.resize(x.double().cpu().numpy(), [dict(r=ratio[0], s=ratio[1], method=m)] * 2)
        tol = 2e-6 if out_dtype == torch.float32 else 1e-2
        assert np.abs(a.double().cpu().numpy() - want).max() <= tol * 255


def test_admission_under_tiny_pool(F):
    # every output is the same size; the pool holds two of them
    rng = np.random.default_rng(2)
    reqs = [(inputs.uint8_pixels((1, 3, 600, 600), 50 + k, device="cuda"), (3, 2), int(rng.integers(0, 3)))
            for k in range(16)]
    one = 3 * 900 * 900 * 4
    with F.Server(2 * one, max_inflight=16, tile_budget_per_step=4, auto_release=True) as sv:
        ids = [sv.submit(x, ratio, m) for x, ratio, m in reqs]
        sv.drain(120_000)
        st = sv.stats()
        assert st["completed"] == len(ids)
        assert st["max_inflight_seen"] <= 2  # admission never overcommits the pool
        assert st["deferred"] > 0  # later requests waited for memory freed by completions


def test_pooled_outputs_are_readable(F):
    reqs = _requests(10, 3)
    with F.Server(256 << 20, max_inflight=8, auto_release=False) as sv:
        ids = [sv.submit(x, ratio, m) for x, ratio, m in reqs]
        sv.drain(60_000)
        assert sorted(sv.poll()) == sorted(ids)
        for rid, (x, ratio, m) in zip(ids, reqs):
            y = sv.result(rid)
            assert torch.equal(y, F.resize(x, [F.Axis(*ratio, m)] * 2))
            sv.release(rid)
        with pytest.raises(F.FCFSError):
            sv.release(ids[0])  # already returned


def test_rejections_timeouts_and_bad_requests(F):
    from paper_2203_10670_gb300 import _native as N

    with F.Server(1 << 20, max_inflight=4) as sv:
        big = inputs.uint8_pixels((1, 3, 1024, 1024), 7, device="cuda")
        with pytest.raises(F.FCFSError) as e:
            sv.submit(big, (3, 2), F.BILINEAR)  # output can never fit the 1 MiB pool
        assert e.value.status == N.FCFS_ERR_NOMEM
        assert sv.stats()["rejected"] == 1
        x = inputs.uint8_pixels((1, 3, 40, 40), 8, device="cuda").float()
        w = torch.ones((3, 3, 3), device="cuda")
        d = F.make_desc(x.shape, [F.Axis(3, 2, F.BILINEAR, 1, w)] * 2, N.FCFS_F32, N.FCFS_F32)
        rid = __import__("ctypes").c_ulonglong()
        rc = sv._lib.fcfs_serve_submit(sv._h, __import__("ctypes").byref(d), x.data_ptr(), None, 0.0,
                                      __import__("ctypes").byref(rid))
        assert rc == N.FCFS_ERR_UNSUPPORTED  # learnable weights are not served
    with F.Server(1 << 30, max_inflight=4, tile_budget_per_step=8) as sv:
        reqs = _requests(40, 4, lo=400, hi=800)
        for x, ratio, m in reqs:
            sv.submit(x, ratio, m)
        try:
            sv.drain(0)  # a zero bound returns at once: a timeout unless the work already finished
        except F.FCFSError as e:
            assert e.status == N.FCFS_ERR_TIMEOUT
        sv.drain(60_000)
        assert sv.stats()["completed"] == 40


def test_output_dtype_must_match_the_server(F):
    # the grouped kernel stores every slot in the server's out_dtype, so a request whose
    # output has another dtype is refused on the host before anything is queued (a BF16
    # buffer given to an FP32 server would otherwise receive stores twice its size)
    import ctypes

    from paper_2203_10670_gb300 import _native as N

    x = inputs.uint8_pixels((1, 3, 48, 64), 9, device="cuda")
    axes = [F.Axis(3, 2, F.BILINEAR)] * 2
    for server_dtype, other in ((torch.float32, torch.bfloat16), (torch.bfloat16, torch.float32)):
        with F.Server(64 << 20, out_dtype=server_dtype, max_inflight=4) as sv:
            y = torch.zeros(F.out_shape(x.shape, axes), device="cuda", dtype=other)
            with pytest.raises(F.FCFSError) as e:
                sv.submit(x, (3, 2), F.BILINEAR, y=y)
            assert e.value.status == N.FCFS_ERR_ARG
            d = F.make_desc(x.shape, axes, N.FCFS_U8, N.FCFS_BF16 if other == torch.bfloat16 else N.FCFS_F32)
            rid = ctypes.c_ulonglong()
            for yp in (None, y.data_ptr()):  # pooled and caller-placed outputs alike
                rc = sv._lib.fcfs_serve_submit(sv._h, ctypes.byref(d), x.data_ptr(), yp, 0.0, ctypes.byref(rid))
                assert rc == N.FCFS_ERR_ARG
            st = sv.stats()
            assert st["submitted"] == 0 and st["steps"] == 0
            torch.cuda.synchronize()
            assert int(torch.count_nonzero(y.float())) == 0  # nothing was written


def test_batch_submission(F):
    # one call queues many requests; results equal the standalone forward; an invalid request
    # stops the batch after the ones before it were queued
    import ctypes

    from paper_2203_10670_gb300 import _native as N

    reqs = _requests(40, 6)
    outs, descs, xs, ys = [], [], [], []
    for x, ratio, m in reqs:
        axes = [F.Axis(*ratio, m)] * 2
        y = torch.empty(F.out_shape(x.shape, axes), device="cuda")
        outs.append(y)
        descs.append(F.make_desc(x.shape, axes, N.FCFS_U8, N.FCFS_F32))
        xs.append(x.data_ptr())
        ys.append(y.data_ptr())
    with F.Server(1 << 30, max_inflight=16, tile_budget_per_step=64) as sv:
        t = F.Server.clock()
        ids = sv.submit_batch_raw(descs, xs, ys, [t] * len(descs))
        assert len(set(ids)) == len(reqs)
        sv.drain(60_000)
        assert sorted(sv.poll()) == sorted(ids)
        # an invalid third request: the first two are queued, its status is returned
        bad = F.make_desc(reqs[0][0].shape, [F.Axis(3, 2, F.BILINEAR)] * 2, N.FCFS_U8, N.FCFS_BF16)
        darr = (N.fcfs_desc * 4)(descs[0], descs[1], bad, descs[3])
        xarr = (ctypes.c_void_p * 4)(*xs[:4])
        yarr = (ctypes.c_void_p * 4)(*ys[:4])
        tarr = (ctypes.c_double * 4)(t, t, t, t)
        idarr = (ctypes.c_ulonglong * 4)()
        n = ctypes.c_int()
        rc = sv._lib.fcfs_serve_submit_batch(sv._h, 4, darr, xarr, yarr, tarr, idarr, ctypes.byref(n))
        assert rc == N.FCFS_ERR_ARG and n.value == 2
        sv.drain(60_000)
        assert sorted(sv.poll()) == sorted(idarr[:2])
    torch.cuda.synchronize()
    for (x, ratio, m), y in zip(reqs, outs):
        assert torch.equal(y, F.resize(x, [F.Axis(*ratio, m)] * 2))


def test_cancel_queued_and_running_requests(F):
    # a client that gives up on requests: queued ones leave at once, running ones stop receiving
    # tiles; every id is still reported once, the rest of the stream completes normally
    # a large first request (thousands of two-tile steps) keeps the others queued behind it while
    # the client cancels: one request admitted at a time
    big = (inputs.uint8_pixels((1, 3, 2048, 2048), 4321, device="cuda"), (3, 2), 2)
    reqs = [big] + _requests(23, 7, lo=400, hi=800)
    with F.Server(1 << 30, max_inflight=1, tile_budget_per_step=2, auto_release=False) as sv:
        ids = [sv.submit(x, ratio, m) for x, ratio, m in reqs]
        victims = set(ids[1::3])
        for rid in ids[1::3]:
            sv.cancel(rid)  # queued: leaves at once
        try:
            sv.cancel(ids[0])  # running (or, on a very fast device, already finished)
            victims.add(ids[0])
        except F.FCFSError:
            pass
        with pytest.raises(F.FCFSError):
            sv.cancel(10 ** 9)  # unknown id
        sv.drain(120_000)
        done = []
        while True:
            got = sv.poll()
            if not got:
                break
            done += got
        assert sorted(done) == sorted(ids)
        st = sv.stats()
        assert st["canceled"] == len(victims) and st["completed"] == len(ids) - len(victims)
        for rid, (x, ratio, m) in zip(ids, reqs):
            if rid in victims:
                with pytest.raises(F.FCFSError):
                    sv.result(rid)  # no output for a canceled request
            else:
                assert torch.equal(sv.result(rid), F.resize(x, [F.Axis(*ratio, m)] * 2))
                sv.release(rid)


def test_device_status_clean_after_serving(F):
    assert F.fcfs_device_status(clear=True) == 0
