"""Serving: continuous batching through tls_serve_* (GPU).

* every job's result is bitwise the same as the same vectors smeared alone
  with the multi-RHS kernel (alone vs in the mix), and within the storage
  tolerance of the FP64 oracle;
* jobs submitted while a long job runs are admitted into the running batch and
  finish first;
* admission by HBM footprint, host buffers, stop with queued jobs, and a gauge
  that is in use cannot be freed.
"""

import numpy as np
import pytest
import torch

import oracle
from helpers import rel_l2
from paper_2301_05518_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2301_05518_gb300 import tls as t
    return t


def _gauge(T, ctx, dims, seed, wprec=None, device=False):
    U = synth.gauge_haar(dims, seed, nd=4)
    gid = ctx.load_gauge(U.cuda() if device else U, 4, dims)
    ctx.build_twolink(gid, wprec if wprec is not None else T.TLS_F32, T.TLS_R18)
    return gid, U


def test_mix_equals_alone_and_oracle(T):
    rng = np.random.default_rng(5)
    with T.Context(0) as ctx:
        dims_a, dims_b = (8, 8, 8, 4), (6, 4, 8, 3)
        ga, Ua = _gauge(T, ctx, dims_a, 41)
        gb, Ub = _gauge(T, ctx, dims_b, 42)
        specs = []
        for k in range(10):
            gid, U, dims = (ga, Ua, dims_a) if k % 2 == 0 else (gb, Ub, dims_b)
            nvec = int(rng.integers(1, 5))
            N = int(rng.integers(2, 12))
            width = float(N * rng.uniform(0.05, 0.3))
            storage = T.TLS_F32 if k % 3 else T.TLS_F16
            t0 = -1 if k % 4 else 1
            vecs = synth.gaussian_vectors(dims, nvec, 100 + k, dtype=torch.complex64)
            specs.append((gid, U, dims, nvec, N, width, storage, t0, vecs))
        ctx.serve_start(max_slots=12, steps_per_launch=3, use_graphs=1)
        jobs = []
        for (gid, U, dims, nvec, N, width, storage, t0, vecs) in specs:
            x = vecs.clone().cuda()
            jobs.append((ctx.serve_submit(gid, x, T.TLS_F32, nvec, N, width, timeslice=t0, storage=storage), x))
        results = [ctx.serve_wait(j, timeout_s=120) for j, _ in jobs]
        ctx.serve_stop()
        for r in results:
            assert r["status"] == 0 and r["done_ms"] >= r["start_ms"] >= r["submit_ms"]
        for (gid, U, dims, nvec, N, width, storage, t0, vecs), (_, x) in zip(specs, jobs):
            alone = vecs.clone().cuda()
            ctx.smear(gid, alone, T.TLS_F32, nvec, N, width, timeslice=t0, storage=storage,
                      kernel=T.TLS_KERNEL_MRHS)
            assert torch.equal(alone, x)
            want = oracle.smear(oracle.twolink(U.numpy()), vecs.numpy().astype(np.complex128), N, width, t0=t0)
            tol = 2e-6 * N if storage == T.TLS_F32 else 5e-3
            got = x.cpu().numpy().astype(np.complex128)
            for v in range(nvec):
                assert rel_l2(got[v], want[v]) <= tol


def test_late_jobs_join_a_running_batch(T):
    with T.Context(0) as ctx:
        dims = (16, 16, 16, 4)
        gid, U = _gauge(T, ctx, dims, 43)
        ctx.serve_start(max_slots=8, steps_per_launch=1, use_graphs=1)
        long_x = synth.gaussian_vectors(dims, 1, 7, dtype=torch.complex64).cuda()
        jl = ctx.serve_submit(gid, long_x, T.TLS_F32, 1, 3000, 300.0)
        short = []
        for k in range(3):
            x = synth.gaussian_vectors(dims, 2, 8 + k, dtype=torch.complex64).cuda()
            short.append((ctx.serve_submit(gid, x, T.TLS_F32, 2, 5, 1.0), x))
        rs = [ctx.serve_wait(j, 120) for j, _ in short]
        rl = ctx.serve_wait(jl, 300)
        ctx.serve_stop()
        assert all(r["done_ms"] < rl["done_ms"] for r in rs)
        # admitted while the long job was on the device
        assert all(r["start_ms"] < rl["done_ms"] for r in rs)


def test_host_buffer_jobs(T):
    with T.Context(0) as ctx:
        dims = (8, 4, 6, 3)
        gid, U = _gauge(T, ctx, dims, 44)
        vecs = synth.gaussian_vectors(dims, 3, 9, dtype=torch.complex64)
        host = vecs.clone()
        ctx.serve_start(max_slots=4)
        j = ctx.serve_submit(gid, host, T.TLS_F32, 3, 6, 1.2, timeslice=2)
        ctx.serve_wait(j, 60)
        ctx.serve_stop()
        dev = vecs.clone().cuda()
        ctx.smear(gid, dev, T.TLS_F32, 3, 6, 1.2, timeslice=2, kernel=T.TLS_KERNEL_MRHS)
        assert torch.equal(dev.cpu(), host)


def test_admission_errors_and_lifecycle(T):
    dims = (8, 8, 8, 4)
    with T.Context(0, hbm_cap_bytes=16 << 20) as ctx:
        gid, U = _gauge(T, ctx, dims, 45)
        ctx.serve_start(max_slots=64)
        x = synth.gaussian_vectors(dims, 2, 10, dtype=torch.complex64).cuda()
        # a 64-slot batch of 8^3x4 FP32 vectors needs 2 x 64 x 49 KB: fits; F64 W is absent
        with pytest.raises(T.TLSError) as e:
            ctx.serve_submit(gid, x, T.TLS_F32, 2, 3, 1.0, storage=T.TLS_F64)
        assert e.value.status == T.TLS_ERR_UNSUPPORTED
        with pytest.raises(T.TLSError) as e:
            ctx.serve_submit(gid, x, T.TLS_F32, 65, 3, 1.0)
        assert e.value.status == T.TLS_ERR_ARG
        j = ctx.serve_submit(gid, x, T.TLS_F32, 2, 3, 1.0)
        ctx.serve_wait(j, 60)
        ctx.serve_stop()
    big = (16, 16, 16, 16)
    with T.Context(0, hbm_cap_bytes=48 << 20) as ctx:
        gid, U = _gauge(T, ctx, big, 46, device=True)
        ctx.serve_start(max_slots=64)
        x = synth.gaussian_vectors(big, 1, 11, dtype=torch.complex64).cuda()
        # 64 slots x 2 buffers x 65536 sites x 24 B = 201 MB > cap: can never fit
        with pytest.raises(T.TLSError) as e:
            ctx.serve_submit(gid, x, T.TLS_F32, 1, 3, 1.0)
        assert e.value.status == T.TLS_ERR_ADMIT
        ctx.serve_stop()


def test_busy_gauge_cannot_be_freed(T):
    with T.Context(0) as ctx:
        dims = (16, 16, 16, 8)
        gid, U = _gauge(T, ctx, dims, 47)
        ctx.serve_start(max_slots=4)
        x = synth.gaussian_vectors(dims, 1, 12, dtype=torch.complex64).cuda()
        # long enough (a few seconds) that the job is still in its batch when free_gauge runs
        j = ctx.serve_submit(gid, x, T.TLS_F32, 1, 100000, 5000.0)
        with pytest.raises(T.TLSError) as e:
            ctx.free_gauge(gid)
        assert e.value.status == T.TLS_ERR_STATE
        ctx.serve_wait(j, 300)
        ctx.serve_stop()
        ctx.free_gauge(gid)
