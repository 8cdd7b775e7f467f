"""The library under concurrent host threads.

Eight Python threads (ctypes releases the interpreter lock for each call)
drive the entry points at once, each on its own CUDA stream with its own
outputs: the staged, LDG, texture and quad back-projections (the last two
share the library's cached staging buffers across streams), the host-buffer
schedule, the batched plan, the adjoint and the pre-processing filter.  Each
thread repeats the same sequence of calls, so every deterministic result
must equal the same sequence run on one thread bit for bit; the adjoint,
whose cross-CTA reductions make its summation order vary, is checked
against the oracle.  Every call's status is checked, and the bounded waits'
status word at the end.
"""
import os
import threading

import numpy as np
import pytest
import torch

import oracle
import synth
from _helpers import assert_parity
from paper_1401_3615_gb300 import fdk

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 1
THREADS = 8
REPS = 4


@pytest.fixture(scope="module")
def scans():
    a = synth.make_scan(synth.preset("small", nx=37, ny=29, nz=21, det_w=64, det_h=48), device="cuda")
    b = synth.make_scan(synth.preset("small", nx=24, ny=30, nz=18, n_views=20, det_w=56, det_h=40,
                                     pixel=0.308 * 1248.0 / 56, seed=5), device="cuda")
    raw = synth.projections(synth.preset("small", n_views=6, det_w=1248, det_h=4, pixel=0.308),
                            filtered=False, device="cuda")
    return a, b, raw


def _zeros(s):
    d = s["dims"]
    return torch.zeros((int(d[2]), int(d[1]), int(d[0])), dtype=torch.float32, device="cuda")


def _sequence(a, b, raw, stream):
    """One thread's calls, REPS times, on ``stream``; returns its outputs."""
    geo_a = (a["mats"], a["voxel_size"], a["origin"])
    geo_b = (b["mats"], b["voxel_size"], b["origin"])
    raw_mats = synth.geometry(synth.preset("small", n_views=6, det_w=1248, det_h=4, pixel=0.308))["mats"]
    with torch.cuda.stream(stream):
        out = {k: _zeros(a) for k in ("stage", "ldg", "tex", "quad")}
        out["batch_a"], out["batch_b"] = _zeros(a), _zeros(b)
        out["adj"] = torch.zeros_like(a["proj"])
        out["filter"] = torch.empty_like(raw)
        host_proj = b["proj"].cpu().pin_memory()
        host_vol = torch.empty(tuple(_zeros(b).shape), dtype=torch.float32).pin_memory()
        x = torch.from_numpy(synth.gaussian_volume(a["dims"], seed=9)).to("cuda")
        plan = fdk.fdk_batch_plan_create([(out["batch_a"], a["proj"], *geo_a), (out["batch_b"], b["proj"], *geo_b)])
        for _ in range(REPS):
            for key, fetch in (("stage", fdk.FETCH_STAGE), ("ldg", fdk.FETCH_LDG), ("tex", fdk.FETCH_TEX),
                               ("quad", fdk.FETCH_QUAD)):
                fdk.fdk_backproject(out[key], a["proj"], *geo_a, fetch=fetch)
            plan.execute()
            fdk.fdk_forwardproject_adjoint(out["adj"], x, *geo_a)
            fdk.fdk_preweight_filter(out["filter"], raw, raw_mats, scale=0.5)
            fdk.fdk_backproject_host(host_vol, host_proj, *geo_b, overwrite=True)
        stream.synchronize()
        plan.close()
    out["host"] = host_vol.clone()
    return out


def test_concurrent_threads(scans):
    a, b, raw = scans
    ref = _sequence(a, b, raw, torch.cuda.Stream())
    fdk.fdk_device_status()
    results, errors = [None] * THREADS, []

    def work(i):
        try:
            results[i] = _sequence(a, b, raw, torch.cuda.Stream())
        except Exception as e:          # reported below, with the thread's index
            errors.append((i, repr(e)))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(THREADS)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not any(t.is_alive() for t in threads), "a thread did not finish"
    assert not errors, errors
    torch.cuda.synchronize()
    fdk.fdk_device_status()
    for i, r in enumerate(results):
        for key in ref:
            if key == "adj":
                continue
            assert torch.equal(r[key], ref[key]), (i, key)
    # the adjoint against the oracle: REPS accumulations of the transpose
    x = synth.gaussian_volume(a["dims"], seed=9)
    W, H = a["proj"].shape[2], a["proj"].shape[1]
    q = oracle.adjoint(x, a["mats"], a["dims"], a["voxel_size"], a["origin"], W, H, threads=NCPU)
    for i, r in enumerate([ref] + results):
        assert_parity(REPS * q, r["adj"].cpu().numpy(), what=f"adjoint, thread {i}")
    # and the deterministic results against the oracle once
    f = oracle.backproject(a["proj"].cpu().numpy(), a["mats"], a["dims"], a["voxel_size"], a["origin"],
                           threads=NCPU)
    for key in ("stage", "ldg", "tex", "quad", "batch_a"):
        assert_parity(REPS * f, ref[key].cpu().numpy(), what=key)
