"""GPU request loop: continuous batching of solve requests (hisq_submit / hisq_poll).

A seeded Poisson-like stream of requests on two lattice volumes, with
different masses and tolerances and some multi-shift requests, is queued at
once; every result's FP64 true residual, recomputed by the CPU oracle, must
meet its own target, and every result must equal the same request solved
alone, bitwise: a CG request's arithmetic does not depend on the batch
session's other slots, its tile or when it joined (it always starts at a
block boundary), and a multi-shift request runs the same kernels on the same
grid whatever else is on the device.  Bounded waits time out cleanly,
unknown tickets and bad requests are refused, and the stats report latency
percentiles and throughput.
"""
import time

import numpy as np
import pytest
import torch

from paper_2302_09224_gb300 import hisq, synth

pytestmark = pytest.mark.gpu

VOLS = [(8, 8, 8, 8), (8, 8, 4, 16)]


@pytest.fixture(scope="module")
def env():
    ctx = hisq.hisq_create(0)
    gauges, fields = {}, {}
    for d in VOLS:
        fat, lng = synth.gauge_pair(d, seed=0)
        fields[d] = (fat.numpy(), lng.numpy())
        gauges[d] = hisq.hisq_load_gauge(ctx, d, fat.cuda(), lng.cuda())
    yield ctx, gauges, fields
    hisq.hisq_destroy(ctx)


def requests(n, seed=1):
    g = np.random.Generator(np.random.Philox(key=seed))
    out = []
    for i in range(n):
        d = VOLS[int(g.integers(len(VOLS)))]
        m = float(np.exp(g.uniform(np.log(0.02), np.log(0.2))))
        tol = [1e-6, 1e-8, 1e-10][int(g.integers(3))]
        ms = bool(g.uniform() < 0.3)
        out.append(dict(dims=d, mass=m, tol=tol, ms=ms, seed=synth.rhs_seed(i)))
    return out


def submit(ctx, gauges, q, on_device=True):
    d = q["dims"]
    b = synth.spinor(d, q["seed"])
    b = b.cuda() if on_device else b.numpy()
    if q["ms"]:
        sig = synth.shifts_logspaced(4, 1e-3, 0.5)
        tols = [q["tol"]] * 4
        x = torch.zeros((4,) + tuple(b.shape), dtype=torch.float64, device="cuda") if on_device else \
            np.zeros((4,) + b.shape)
        t = hisq.hisq_submit(ctx, gauges[d], hisq.HISQ_REQ_MULTISHIFT, q["mass"], b, x, on_device, sigma=sig,
                             shift_tol=tols)
        return t, b, x, sig
    x = torch.zeros_like(b) if on_device else np.zeros_like(b)
    t = hisq.hisq_submit(ctx, gauges[d], hisq.HISQ_REQ_CG, q["mass"], b, x, on_device, tol=q["tol"])
    return t, b, x, None


def as_np(a):
    return a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)


def test_stream_in_the_mix_matches_alone(env, orc):
    ctx, gauges, fields = env
    qs = requests(24)
    live = [(q, *submit(ctx, gauges, q, on_device=(i % 3 != 0))) for i, q in enumerate(qs)]
    results = {}
    for q, t, b, x, sig in live:
        st, info = hisq.hisq_wait(ctx, t, 120.0)
        assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
        results[t] = (q, b, x, sig)
    for t, (q, b, x, sig) in results.items():
        d = q["dims"]
        fat, lng = fields[d]
        bb = as_np(b)
        xx = as_np(x)
        if sig is None:
            r = bb - orc.mee(d, fat, lng, q["mass"], xx)
            assert np.linalg.norm(r) / np.linalg.norm(bb) <= q["tol"]
        else:
            for i, s in enumerate(sig):
                r = bb - orc.mee(d, fat, lng, q["mass"], xx[i], sigma=s)
                assert np.linalg.norm(r) / np.linalg.norm(bb) <= q["tol"]
    # every request again, alone: the same bits, shift by shift for multi-shift
    n_cg = n_ms = 0
    for t, (q, b, x, sig) in results.items():
        t2, b2, x2, _ = submit(ctx, gauges, q)
        st, _ = hisq.hisq_wait(ctx, t2, 120.0)
        assert st == hisq.HISQ_OK
        alone, mixed = as_np(x2), as_np(x)
        if sig is None:
            n_cg += 1
            np.testing.assert_array_equal(alone, mixed)
        else:
            n_ms += 1
            for i in range(len(sig)):
                np.testing.assert_array_equal(alone[i], mixed[i])
    assert n_cg > 0 and n_ms > 0
    s = hisq.hisq_serve_stats(ctx)
    assert s.completed >= 24 and s.latency_p99_s >= s.latency_p50_s > 0 and s.solves_per_s > 0


def test_wait_timeout_poll_and_refusals(env):
    ctx, gauges, fields = env
    q = dict(dims=VOLS[0], mass=0.02, tol=1e-10, ms=False, seed=5)
    t, b, x, _ = submit(ctx, gauges, q)
    try:
        hisq.hisq_wait(ctx, t, 0.0)
    except hisq.HisqError as e:
        assert e.status == hisq.HISQ_ETIMEOUT
    st, info = hisq.hisq_wait(ctx, t, 60.0)
    assert st == hisq.HISQ_OK and info.true_residual <= 1e-10
    with pytest.raises(hisq.HisqError, match="ENOTFOUND"):
        hisq.hisq_poll(ctx, t)
    t2, b2, x2, _ = submit(ctx, gauges, q)
    done = False
    for _ in range(2000):
        done, st, info = hisq.hisq_poll(ctx, t2)
        if done:
            break
        time.sleep(0.005)
    assert done and st == hisq.HISQ_OK
    with pytest.raises(hisq.HisqError, match="EINVAL"):
        hisq.hisq_submit(ctx, gauges[VOLS[0]], 7, 0.1, b, x, True)


def test_admission_by_budget():
    """A context whose HBM budget holds the resident gauge fields, the workers'
    reduction lanes and about one batch session at a time: sessions that do not
    fit wait for memory to free up instead of failing, every request finishes
    OK with the same bits as on an unconstrained context, and the context never
    holds more than its budget."""
    big = hisq.hisq_create(0)
    d = VOLS[0]
    fat, lng = synth.gauge_pair(d, seed=0)
    qs = [dict(dims=d, mass=m, tol=1e-10, ms=False, seed=synth.rhs_seed(40 + i))
          for i, m in enumerate([0.05, 0.1, 0.03, 0.2, 0.08, 0.04, 0.15, 0.06, 0.12, 0.09])]
    try:
        gb = {d: hisq.hisq_load_gauge(big, d, fat.cuda(), lng.cuda())}
        ref = [submit(big, gb, q) for q in qs]
        for t, b, x, _ in ref:
            assert hisq.hisq_wait(big, t, 120.0)[0] == hisq.HISQ_OK
        # resident fields and their stored copies, measured on a warm context
        probe = hisq.hisq_create(0)
        g0 = hisq.hisq_load_gauge(probe, d, fat.cuda(), lng.cuda())
        b0 = synth.spinor(d, 1).cuda()
        p = hisq.hisq_default_params()
        p.mass, p.on_device = 0.1, 1
        hisq.hisq_cg(probe, g0, p, b0, torch.zeros_like(b0))
        resident = hisq.hisq_mem_used(probe)
        hisq.hisq_destroy(probe)
        lane = 8 * ((1 << 16) * 32 + 32) + 256 + 4 * (32 + 4096)
        budget = resident + 2 * lane + (6 << 20)   # two workers, room for about one 8-slot session of 8^4
        small = hisq.hisq_create(0, budget)
        try:
            gs = {d: hisq.hisq_load_gauge(small, d, fat.cuda(), lng.cuda())}
            # each request on its own key (maxiter differs), so the sessions compete for memory
            live = []
            for i, q in enumerate(qs):
                b = synth.spinor(d, q["seed"]).cuda()
                x = torch.zeros_like(b)
                t = hisq.hisq_submit(small, gs[d], hisq.HISQ_REQ_CG, q["mass"], b, x, True, tol=q["tol"],
                                     maxiter=100000 - i)
                live.append((t, b, x))
            peak = 0
            for t, b, x in live:
                while True:
                    peak = max(peak, hisq.hisq_mem_used(small))
                    done, st, _ = hisq.hisq_poll(small, t)
                    if done:
                        assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
                        break
                    time.sleep(0.002)
            assert peak <= budget
            for (t, b, x), (_, _, xr, _) in zip(live, ref):
                np.testing.assert_array_equal(as_np(x), as_np(xr))
        finally:
            hisq.hisq_destroy(small)
    finally:
        hisq.hisq_destroy(big)


def test_multishift_refinement_paths(env, orc):
    """A multi-shift request's refinements in a triplet with batch sessions (20-bit) and in one without
    (30-bit, FP64-class: the single-system CG from the stage's solution), both from host and device
    buffers: every shift meets its target by the oracle's FP64 residual, refinements ran where the
    stage left a shift above its target, and the report is in the caller's shift order."""
    ctx, gauges, fields = env
    d = VOLS[0]
    fat, lng = fields[d]
    sig = [0.3, 1e-3, 0.05, 0.01]  # unsorted on purpose
    tols = [1e-10, 1e-10, 1e-9, 1e-10]
    for refine, on_device in (("int20", True), ("int30", False)):
        b = synth.spinor(d, synth.rhs_seed(77))
        bb = b.numpy()
        bx = b.cuda() if on_device else bb
        x = torch.zeros((4,) + tuple(b.shape), dtype=torch.float64, device="cuda") if on_device else \
            np.zeros((4,) + bb.shape)
        t = hisq.hisq_submit(ctx, gauges[d], hisq.HISQ_REQ_MULTISHIFT, 0.02, bx, x, on_device, sigma=sig,
                             shift_tol=tols, sloppy=hisq.prec("half"), refine=hisq.prec(refine, 18 if refine == "int30" else 12))
        st, info = hisq.hisq_wait(ctx, t, 120.0)
        assert st == hisq.HISQ_OK, hisq.STATUS_NAMES[st]
        xx = as_np(x)
        for i, s in enumerate(sig):
            r = bb - orc.mee(d, fat, lng, 0.02, xx[i], sigma=s)
            assert np.linalg.norm(r) / np.linalg.norm(bb) <= tols[i], (refine, i)
            assert info.shift_resid[i] <= tols[i]
        assert sum(info.refine_iters[i] for i in range(4)) > 0
        assert info.shift_resid_ms[1] >= info.shift_resid[1]  # the lightest shift was refined
