"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative L2 per vector against the FP64 oracle):
  FP64 storage        <= 1e-13
  FP32 storage        <= 2e-6 * N   (raw error / N <= 2e-6)
  FP16/BF16 storage   <= 5e-3
Index maps (ingest, sublattice decoupling, untouched slices) are bit-exact.
"""

import numpy as np
import pytest
import torch

import oracle
from helpers import per_vector_rel_l2, rel_l2, sublattice_mask
from paper_2301_05518_gb300 import synth, workloads

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module")
def T():
    from paper_2301_05518_gb300 import tls as t
    return t


@pytest.fixture(scope="module")
def ctx(T):
    c = T.Context(0)
    yield c
    c.close()


def tol(storage, N):
    from paper_2301_05518_gb300 import tls as t
    if storage == t.TLS_F64:
        return 1e-13
    if storage == t.TLS_F32:
        return 2e-6 * max(N, 1)
    return 5e-3


def gauge_dev(dims, kind, seed, eps=0.3, nd=4):
    if kind == "haar":
        return synth.gauge_haar(dims, seed, nd=nd, device="cuda")
    return synth.gauge_near_unit(dims, eps, seed, nd=nd, device="cuda")


_ORACLE_CACHE = {}


def cached(key, fn):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = fn()
    return _ORACLE_CACHE[key]


def gauge(dims, kind, seed, eps=0.3, nd=4):
    if kind == "haar":
        return synth.gauge_haar(dims, seed, nd=nd)
    if kind == "unit":
        return synth.gauge_unit(dims, nd=nd)
    return synth.gauge_near_unit(dims, eps, seed, nd=nd)


# ------------------------------------------------------------------ ingest
@pytest.mark.parametrize("dims", [(4, 6, 8, 3), (2, 2, 2, 1), (6, 10, 4, 2), (8, 8, 8, 2)])
@pytest.mark.parametrize("nd,on_device", [(4, False), (3, True), (4, "pinned")])
def test_ingest_roundtrip_bit_exact(ctx, T, dims, nd, on_device):
    U = gauge(dims, "haar", 5, nd=nd)
    src = U.pin_memory() if on_device == "pinned" else (U.cuda() if on_device else U)
    gid = ctx.load_gauge(src, nd, dims)
    out = np.zeros(U.shape[:4] + (3, 3, 3), dtype=np.complex128)
    ctx.export_gauge(gid, out)
    assert np.array_equal(out, U.numpy()[..., :3, :, :])
    ctx.free_gauge(gid)


# ------------------------------------------------------------------ build
BUILD_CASES = [("F64", 18, 1e-15), ("F32", 18, 4e-7), ("F32", 12, 1e-6), ("F32", 8, 3e-6),
               ("F16", 18, 6e-4), ("F16", 12, 2e-3), ("BF16", 18, 5e-3), ("BF16", 12, 1.5e-2)]


@pytest.mark.parametrize("prec,recon,bound", BUILD_CASES)
def test_build_matches_oracle(ctx, T, prec, recon, bound):
    dims = (6, 4, 8, 3)
    U = gauge(dims, "haar", 7)
    want = oracle.twolink(U.numpy())
    gid = ctx.load_gauge(U, 4, dims)
    ctx.build_twolink(gid, getattr(T, "TLS_" + prec), recon)
    got = np.zeros_like(want)
    ctx.export_twolink(gid, got)
    assert np.abs(got - want).max() <= bound
    ctx.free_gauge(gid)


def test_build_recon8_rejects_identity(ctx, T):
    dims = (4, 4, 4, 1)
    gid = ctx.load_gauge(gauge(dims, "unit", 0), 4, dims)
    with pytest.raises(T.TLSError) as e:
        ctx.build_twolink(gid, T.TLS_F32, T.TLS_R8)
    assert e.value.status == T.TLS_ERR_DEVICE
    ctx.build_twolink(gid, T.TLS_F32, T.TLS_R12)  # the context stays usable
    ctx.free_gauge(gid)


# ------------------------------------------------------------------ smearing parity
def _run(ctx, T, U, dims, vecs, storage, wprec, recon, kernel, N, sigma, t0, io=None, host=False):
    gid = ctx.load_gauge(U, U.shape[4], dims)
    ctx.build_twolink(gid, wprec, recon)
    io = io if io is not None else (T.TLS_F64 if storage == T.TLS_F64 else T.TLS_F32)
    dt = torch.complex128 if io == T.TLS_F64 else torch.complex64
    x = vecs.to(dt).contiguous()
    x = (x.pin_memory() if host == "pinned" else x) if host else x.cuda()
    norms = ctx.smear(gid, x, io, x.shape[0], N, sigma, timeslice=t0, storage=storage, kernel=kernel,
                      norms=True)
    ctx.free_gauge(gid)
    return x.cpu().numpy().astype(np.complex128), norms


SMEAR_CASES = [
    # storage, W prec, recon, kernels
    ("F64", "F64", 18, ("SINGLE", "MRHS", "PERSISTENT")),
    ("F32", "F32", 18, ("SINGLE", "MRHS", "PERSISTENT")),
    ("F32", "F32", 12, ("MRHS", "PERSISTENT")),
    ("F32", "F32", 8, ("MRHS", "PERSISTENT")),
    ("F16", "F32", 18, ("MRHS", "PERSISTENT")),
    ("F16", "F16", 12, ("MRHS", "PERSISTENT")),
    ("F16", "F16", 18, ("SINGLE",)),
    ("BF16", "F32", 12, ("MRHS", "PERSISTENT")),
    ("BF16", "BF16", 18, ("MRHS",)),
]


@pytest.mark.parametrize("storage,wprec,recon,kernels", SMEAR_CASES)
@pytest.mark.parametrize("t0", [-1, 1])
def test_smear_matches_oracle(ctx, T, storage, wprec, recon, kernels, t0):
    dims = (6, 4, 8, 3)
    U = gauge(dims, "haar", 11)
    vecs = synth.gaussian_vectors(dims, 5, 12)
    N, sigma = 7, 1.4
    want = oracle.smear(oracle.twolink(U.numpy()), vecs.numpy(), N, sigma, t0=t0)
    st = getattr(T, "TLS_" + storage)
    for kname in kernels:
        got, norms = _run(ctx, T, U, dims, vecs, st, getattr(T, "TLS_" + wprec), recon,
                          getattr(T, "TLS_KERNEL_" + kname), N, sigma, t0)
        errs = per_vector_rel_l2(got, want)
        assert max(errs) <= tol(st, N), (kname, errs)
        # untouched slices are bit-exact copies (within the io precision)
        if t0 >= 0:
            io_in = vecs.numpy() if st == T.TLS_F64 else vecs.to(torch.complex64).numpy().astype(np.complex128)
            for t in range(dims[3]):
                if t != t0:
                    assert np.array_equal(got[:, t], io_in[:, t])
        sl = slice(None) if t0 < 0 else slice(t0, t0 + 1)
        ref_norms = (np.abs(got[:, sl]) ** 2).reshape(got.shape[0], -1).sum(1)
        assert np.allclose(norms, ref_norms, rtol=1e-12, atol=0)


def test_io_f64_with_f32_storage(ctx, T):
    dims = (4, 4, 6, 2)
    U = gauge(dims, "near", 13)
    vecs = synth.gaussian_vectors(dims, 3, 14)
    N, sigma = 5, 1.0
    want = oracle.smear(oracle.twolink(U.numpy()), vecs.numpy(), N, sigma)
    got, _ = _run(ctx, T, U, dims, vecs, T.TLS_F32, T.TLS_F32, 18, T.TLS_KERNEL_MRHS, N, sigma, -1,
                  io=T.TLS_F64)
    assert max(per_vector_rel_l2(got, want)) <= 2e-6 * N


@pytest.mark.parametrize("storage", ["F64", "F32", "F16"])
def test_mrhs_bitwise_equals_single_vector(ctx, T, storage):
    """A vector's result does not depend on nvec or on the other vectors in the batch."""
    dims = (8, 4, 6, 2)
    U = gauge(dims, "haar", 15)
    vecs = synth.gaussian_vectors(dims, 6, 16)
    st = getattr(T, "TLS_" + storage)
    wp = T.TLS_F64 if st == T.TLS_F64 else T.TLS_F32
    batch, _ = _run(ctx, T, U, dims, vecs, st, wp, 18, T.TLS_KERNEL_MRHS, 6, 1.3, -1)
    single, _ = _run(ctx, T, U, dims, vecs, st, wp, 18, T.TLS_KERNEL_SINGLE, 6, 1.3, -1)
    assert np.array_equal(batch, single)
    alone, _ = _run(ctx, T, U, dims, vecs[3:4], st, wp, 18, T.TLS_KERNEL_MRHS, 6, 1.3, -1)
    assert np.array_equal(alone[0], batch[3])
    p_batch, _ = _run(ctx, T, U, dims, vecs, st, wp, 18, T.TLS_KERNEL_PERSISTENT, 6, 1.3, -1)
    p_alone, _ = _run(ctx, T, U, dims, vecs[2:3], st, wp, 18, T.TLS_KERNEL_PERSISTENT, 6, 1.3, -1)
    assert np.array_equal(p_alone[0], p_batch[2])


@pytest.mark.parametrize("storage", ["F64", "F32"])
def test_zero_steps_and_zero_width_are_identity(ctx, T, storage):
    dims = (4, 4, 4, 2)
    U = gauge(dims, "haar", 17)
    vecs = synth.gaussian_vectors(dims, 2, 18)
    st = getattr(T, "TLS_" + storage)
    wp = T.TLS_F64 if st == T.TLS_F64 else T.TLS_F32
    ref = vecs.numpy() if st == T.TLS_F64 else vecs.to(torch.complex64).numpy().astype(np.complex128)
    for kern in (T.TLS_KERNEL_MRHS, T.TLS_KERNEL_PERSISTENT):
        got, _ = _run(ctx, T, U, dims, vecs, st, wp, 18, kern, 0, 2.0, -1)
        assert np.array_equal(got, ref)
        got, _ = _run(ctx, T, U, dims, vecs, st, wp, 18, kern, 4, 0.0, -1)
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("kern", ["MRHS", "SINGLE", "MRHS_ROWS"])
def test_host_buffers_match_device(ctx, T, kern):
    """Pageable host vectors (staged copies) and pinned ones (read by the kernels over C2C)."""
    dims = (8, 6, 4, 3)
    U = gauge(dims, "near", 19)
    vecs = synth.gaussian_vectors(dims, 3, 20)
    k = getattr(T, "TLS_KERNEL_" + kern)
    for t0 in (-1, 2):
        dev, nd = _run(ctx, T, U, dims, vecs, T.TLS_F32, T.TLS_F32, 18, k, 5, 1.0, t0)
        host, nh = _run(ctx, T, U, dims, vecs, T.TLS_F32, T.TLS_F32, 18, k, 5, 1.0, t0, host=True)
        pinned, npn = _run(ctx, T, U, dims, vecs, T.TLS_F32, T.TLS_F32, 18, k, 5, 1.0, t0, host="pinned")
        assert np.array_equal(dev, host)
        assert np.array_equal(dev, pinned)
        assert np.array_equal(nd, nh) and np.array_equal(nd, npn)


@pytest.mark.parametrize("kern,storage,nvec", [("MRHS", "F32", 5), ("SINGLE", "F32", 2), ("PERSISTENT", "F32", 3),
                                                ("MRHS", "F16", 4), ("MRHS", "F64", 3)])
def test_host_pipeline_slice_groups(ctx, T, kern, storage, nvec):
    """Host vectors through the slice-group pipeline (7 slices: 4 groups of 2, 2, 2, 1 slices in
    three rotating staging slots, copies overlapping the smearing) == device vectors, bitwise,
    norms included; also for one slice."""
    dims = (8, 4, 6, 7)
    U = gauge(dims, "haar", 23)
    vecs = synth.gaussian_vectors(dims, nvec, 24)
    st = getattr(T, "TLS_" + storage)
    wp = T.TLS_F64 if storage == "F64" else T.TLS_F32
    k = getattr(T, "TLS_KERNEL_" + kern)
    for t0 in (-1, 5):
        dev, nd = _run(ctx, T, U, dims, vecs, st, wp, 18, k, 4, 1.1, t0)
        host, nh = _run(ctx, T, U, dims, vecs, st, wp, 18, k, 4, 1.1, t0, host="pinned")
        assert np.array_equal(dev, host)
        assert np.array_equal(nd, nh)


def test_host_gauge_load_two_slots(ctx, T):
    """A host gauge field of more than one staging slot (20 slices of 32^3: the spatial links
    copied by 2-D copies in groups through two slots) ingests bit-exactly."""
    dims = (32, 32, 32, 20)
    U = synth.gauge_haar(dims, 25, nd=4)
    gid = ctx.load_gauge(U, 4, dims)
    out = np.zeros(U.shape[:4] + (3, 3, 3), dtype=np.complex128)
    ctx.export_gauge(gid, out)
    ctx.free_gauge(gid)
    assert np.array_equal(out, U.numpy()[..., :3, :, :])


def test_two_site_extent(ctx, T):
    """L = 2 in every direction: the hop returns to the same site through W and W^dag."""
    dims = (2, 2, 2, 2)
    U = gauge(dims, "haar", 21)
    vecs = synth.gaussian_vectors(dims, 2, 22)
    want = oracle.smear(oracle.twolink(U.numpy()), vecs.numpy(), 5, 1.5)
    for kern in (T.TLS_KERNEL_MRHS, T.TLS_KERNEL_PERSISTENT):
        got, _ = _run(ctx, T, U, dims, vecs, T.TLS_F64, T.TLS_F64, 18, kern, 5, 1.5, -1)
        assert rel_l2(got, want) <= 1e-13


# ------------------------------------------------------------------ errors
def test_error_paths(ctx, T):
    dims = (4, 4, 4, 2)
    U = gauge(dims, "haar", 23)
    with pytest.raises(T.TLSError) as e:
        ctx.load_gauge(U[:, :, :, :3].contiguous(), 4, (3, 4, 4, 2))
    assert e.value.status == T.TLS_ERR_ARG
    gid = ctx.load_gauge(U, 4, dims)
    x = synth.gaussian_vectors(dims, 1, 1).to(torch.complex64).cuda()
    with pytest.raises(T.TLSError) as e:
        ctx.smear(gid, x, T.TLS_F32, 1, 3, 1.0)
    assert e.value.status == T.TLS_ERR_NOT_BUILT
    ctx.build_twolink(gid, T.TLS_F32, 18)
    for kwargs, code in [(dict(N=-1), T.TLS_ERR_ARG), (dict(timeslice=2), T.TLS_ERR_ARG),
                         (dict(storage=T.TLS_F64), T.TLS_ERR_UNSUPPORTED)]:
        args = dict(N=3, timeslice=-1, storage=T.TLS_F32)
        args.update(kwargs)
        with pytest.raises(T.TLSError) as e:
            ctx.smear(gid, x, T.TLS_F32, 1, args["N"], 1.0, timeslice=args["timeslice"],
                      storage=args["storage"])
        assert e.value.status == code
    ctx.free_gauge(gid)
    with pytest.raises(T.TLSError) as e:
        ctx.smear(gid, x, T.TLS_F32, 1, 3, 1.0)
    assert e.value.status == T.TLS_ERR_NOT_FOUND


def test_hbm_cap_admission(T):
    dims = (8, 8, 8, 4)
    with T.Context(0, hbm_cap_bytes=8 << 20) as c:
        U = gauge(dims, "haar", 24)
        gid = c.load_gauge(U, 4, dims)          # 8^3*4 * 3 * 144 B = 884 KB
        c.build_twolink(gid, T.TLS_F32, 18)
        x = synth.gaussian_vectors(dims, 200, 2).to(torch.complex64).cuda()  # ~ 2 x 9.8 MB packed
        with pytest.raises(T.TLSError) as e:
            c.smear(gid, x, T.TLS_F32, 200, 2, 1.0)
        assert e.value.status == T.TLS_ERR_ADMIT
        assert c.bytes_in_use() <= 8 << 20
        c.smear(gid, x[:2].contiguous(), T.TLS_F32, 2, 2, 1.0)  # still usable


def test_barrier_timeout_returns_status(ctx, T):
    """A barrier budget of one poll makes the waits run out; the context stays usable."""
    dims = (16, 16, 16, 2)
    U = gauge(dims, "near", 25)
    vecs = synth.gaussian_vectors(dims, 1, 26)
    gid = ctx.load_gauge(U, 4, dims)
    ctx.build_twolink(gid, T.TLS_F32, 18)
    x = vecs.to(torch.complex64).cuda()
    ctx.set_barrier_budget(1)
    try:
        with pytest.raises(T.TLSError) as e:
            ctx.smear(gid, x, T.TLS_F32, 1, 20, 4.0, kernel=T.TLS_KERNEL_PERSISTENT)
        assert e.value.status == T.TLS_ERR_TIMEOUT
    finally:
        ctx.set_barrier_budget(0)
    x = vecs.to(torch.complex64).cuda()
    ctx.smear(gid, x, T.TLS_F32, 1, 20, 4.0, kernel=T.TLS_KERNEL_PERSISTENT)
    want = oracle.smear(oracle.twolink(U.numpy()), vecs.numpy(), 20, 4.0)
    assert rel_l2(x.cpu().numpy().astype(np.complex128), want) <= 2e-6 * 20
    ctx.free_gauge(gid)


# ------------------------------------------------------------------ the named workloads
def test_small_point_source_workload(ctx, T):
    w = workloads.SMALL_POINT
    dims = w["dims"]
    U = gauge(dims, "near", w["gauge_seed"], eps=w["eps"])
    psi = synth.point_sources(dims, [(0, 0, 0, 0)], [0])
    want = oracle.smear(oracle.twolink(U.numpy()), psi.numpy(), w["N"], w["sigma"], t0=w["timeslice"])
    for kern in (T.TLS_KERNEL_SINGLE, T.TLS_KERNEL_MRHS, T.TLS_KERNEL_PERSISTENT):
        got, _ = _run(ctx, T, U, dims, psi, T.TLS_F64, T.TLS_F64, 18, kern, w["N"], w["sigma"],
                      w["timeslice"])
        assert rel_l2(got, want) <= 1e-13
        assert np.all(got[0, 1:] == 0)
        mask = sublattice_mask(dims, 0)
        assert np.all(got[0, 0][~mask] == 0)


@pytest.mark.parametrize("storage", ["F64", "F32"])
def test_medium_mixed_workload(ctx, T, storage):
    w = workloads.MEDIUM_MIXED
    dims = w["dims"]
    U = cached("medium_U", lambda: gauge_dev(dims, "near", w["gauge_seed"], eps=w["eps"]).cpu())
    pts = synth.point_sources(dims, [(0, 0, 0, 0)] * 3, [0, 1, 2])
    gs = synth.gaussian_vectors(dims, 3, w["vec_seed"])
    def ref():
        W = oracle.twolink(U.numpy())
        return np.concatenate([oracle.smear(W, pts.numpy(), w["N"], w["sigma"], t0=0),
                               oracle.smear(W, gs.numpy(), w["N"], w["sigma"])])
    want = cached("medium", ref)
    st = getattr(T, "TLS_" + storage)
    got, _ = _run(ctx, T, U, dims, torch.cat([pts, gs]), st, st, 18, T.TLS_KERNEL_SINGLE, w["N"],
                  w["sigma"], -1)
    errs = per_vector_rel_l2(got, want)
    assert max(errs) <= tol(st, w["N"]), errs


@pytest.mark.parametrize("storage,wprec,recon", [("F32", "F32", 18), ("F32", "F32", 8),
                                                 ("F16", "F16", 12), ("BF16", "F32", 12)])
def test_large_mrhs_workload_sampled(ctx, T, storage, wprec, recon):
    """48^3x64 Haar, a batch of 12 on the device, checked on two sampled (vector, slice) pairs."""
    w = workloads.LARGE_MRHS
    dims = w["dims"]
    U = gauge_dev(dims, "haar", w["gauge_seed"], nd=3)
    vecs = synth.gaussian_vectors(dims, 12, w["vec_seed"], dtype=torch.complex64, device="cuda")
    st = getattr(T, "TLS_" + storage)
    gid = ctx.load_gauge(U, 3, dims)
    ctx.build_twolink(gid, getattr(T, "TLS_" + wprec), recon)
    ref = {(v, t): vecs[v, t:t + 1].cpu().numpy().astype(np.complex128) for v, t in ((0, 0), (7, 41))}
    ctx.smear(gid, vecs, T.TLS_F32, 12, w["N"], w["sigma"], storage=st, kernel=T.TLS_KERNEL_MRHS)
    ctx.free_gauge(gid)
    for (v, t), src in ref.items():
        want = oracle.smear(oracle.twolink(U[t:t + 1].cpu().numpy()), src, w["N"], w["sigma"])
        got = vecs[v, t:t + 1].cpu().numpy().astype(np.complex128)
        assert rel_l2(got, want) <= tol(st, w["N"])


def test_autotune_picks_a_working_kernel(ctx, T):
    dims = (8, 8, 8, 4)
    U = gauge(dims, "haar", 27)
    vecs = synth.gaussian_vectors(dims, 5, 28, dtype=torch.complex64)
    gid = ctx.load_gauge(U, 4, dims)
    ctx.build_twolink(gid, T.TLS_F32, 18)
    best, cands = ctx.autotune(gid, 5, T.TLS_F32, T.TLS_ALL_T, steps=3)
    assert len(cands) >= 3 and best["ms_per_step"] == min(c["ms_per_step"] for c in cands)
    kinds = {c["kernel"] for c in cands}
    assert T.TLS_KERNEL_MRHS in kinds and T.TLS_KERNEL_PERSISTENT not in kinds  # retired from the tuner
    assert any(tuple(c["tile"])[1] == 6 for c in cands)  # the TMA row kernel is a candidate
    x = vecs.clone().cuda()
    ctx.set_profiling(True)
    ctx.smear(gid, x, T.TLS_F32, 5, 6, 1.2)  # AUTO uses the table entry
    assert ctx.get_profile()["kernel"] == best["kernel"]
    ctx.set_profiling(False)
    want = oracle.smear(oracle.twolink(U.numpy()), vecs.numpy().astype(np.complex128), 6, 1.2)
    assert max(per_vector_rel_l2(x.cpu().numpy().astype(np.complex128), want)) <= 2e-6 * 6
    ctx.free_gauge(gid)


@pytest.mark.parametrize("nvec", [1, 7, 24, 300])
def test_interleaved_groups_bitwise_equal_planar(ctx, T, nvec):
    """Multi-RHS (interleaved, groups of <= 256 vectors) == one vector per launch, bitwise."""
    dims = (4, 6, 4, 2)
    U = gauge(dims, "haar", 29)
    vecs = synth.gaussian_vectors(dims, nvec, 30, dtype=torch.complex64)
    a, na = _run(ctx, T, U, dims, vecs, T.TLS_F32, T.TLS_F32, 12, T.TLS_KERNEL_MRHS, 4, 0.9, -1)
    b, nb = _run(ctx, T, U, dims, vecs, T.TLS_F32, T.TLS_F32, 12, T.TLS_KERNEL_SINGLE, 4, 0.9, -1)
    assert np.array_equal(a, b)
    assert np.array_equal(na, nb)


@pytest.mark.parametrize("kname", ["MRHS_ROWS", "MRHS_ZM"])
@pytest.mark.parametrize("dims,nvec,storage", [((8, 8, 8, 3), 5, "F32"), ((16, 8, 8, 2), 24, "F32"),
                                               ((8, 16, 24, 2), 6, "F16"), ((8, 8, 8, 2), 3, "BF16"),
                                               ((6, 4, 8, 2), 4, "F32"), ((8, 4, 4, 1), 300, "F32"),
                                               ((24, 8, 8, 1), 2, "F16"), ((4, 4, 2, 2), 6, "F32"),
                                               ((2, 2, 2, 1), 2, "F32")])
def test_rows_and_zm_kernels_bitwise_equal_single(ctx, T, kname, dims, nvec, storage):
    """TMA row-staged and z-marching multi-RHS kernels == one vector per launch, bitwise.

    The row kernel falls back to the interleaved kernel when hx % 4 != 0; the
    shapes include hz = 1 and hz = 2 (z-window wrap) and L = 2.
    """
    U = gauge(dims, "haar", 31)
    vecs = synth.gaussian_vectors(dims, nvec, 32, dtype=torch.complex64)
    st = getattr(T, "TLS_" + storage)
    kk = getattr(T, "TLS_KERNEL_" + kname)
    for t0 in (-1, 1 if dims[3] > 1 else 0):
        a, na = _run(ctx, T, U, dims, vecs, st, T.TLS_F32, 18, kk, 5, 1.1, t0)
        b, nb = _run(ctx, T, U, dims, vecs, st, T.TLS_F32, 18, T.TLS_KERNEL_SINGLE, 5, 1.1, t0)
        assert np.array_equal(a, b)
        assert np.array_equal(na, nb)
    if storage == "F32":
        want = oracle.smear(oracle.twolink(U.numpy()), vecs.numpy().astype(np.complex128), 5, 1.1)
        a, _ = _run(ctx, T, U, dims, vecs, st, T.TLS_F32, 18, kk, 5, 1.1, -1)
        assert max(per_vector_rel_l2(a, want)) <= 2e-6 * 5


def test_rows_kernel_at_headline_shape_sampled(ctx, T):
    """64^3 slices with 24 vectors (the headline row shape) on 2 slices vs the oracle."""
    dims = (64, 64, 64, 2)
    U = gauge_dev(dims, "near", 33, eps=0.2)
    vecs = synth.gaussian_vectors(dims, 24, 34, dtype=torch.complex64, device="cuda")
    gid = ctx.load_gauge(U, 4, dims)
    ctx.build_twolink(gid, T.TLS_F32, 18)
    ref = {v: vecs[v, 1:2].cpu().numpy().astype(np.complex128) for v in (0, 13, 23)}
    ctx.smear(gid, vecs, T.TLS_F32, 24, 8, 1.6, storage=T.TLS_F32, kernel=T.TLS_KERNEL_MRHS_ROWS)
    ctx.free_gauge(gid)
    W = oracle.twolink(U[1:2].cpu().numpy())
    for v, src in ref.items():
        want = oracle.smear(W, src, 8, 1.6)
        assert rel_l2(vecs[v, 1:2].cpu().numpy().astype(np.complex128), want) <= 2e-6 * 8


@pytest.mark.parametrize("tile,vb,storage", [((2, 0, 0), 2, "F32"), ((5, 0, 0), 1, "F32"), ((8, 0, 0), 4, "F32"),
                                             ((3, 0, 0), 2, "F32"), ((0, 1, 0), 2, "F32"), ((5, 1, 0), 4, "F32"),
                                             ((3, 1, 0), 1, "F32"), ((0, 2, 0), 2, "F32"), ((5, 2, 0), 4, "F32"),
                                             ((3, 2, 0), 1, "F32"), ((0, 2, 0), 2, "F16"), ((4, 2, 0), 4, "BF16"),
                                             ((7, 2, 0), 1, "F16"), ((0, 3, 0), 2, "F32"), ((5, 3, 0), 4, "F16"),
                                             ((3, 3, 0), 1, "F32"), ((0, 3, 0), 4, "BF16"), ((0, 4, 0), 2, "F32"),
                                             ((5, 4, 0), 4, "F16"), ((3, 4, 0), 1, "BF16"), ((0, 4, 0), 4, "F32"),
                                             ((0, 2, 0), 8, "F32"), ((3, 2, 0), 8, "F32"), ((0, 5, 0), 4, "F32"),
                                             ((0, 5, 0), 2, "F16"), ((5, 5, 0), 1, "BF16"),
                                             ((0, 6, 0), 4, "F32"), ((0, 6, 0), 2, "F32"), ((0, 6, 0), 1, "F32"),
                                             ((4, 6, 0), 4, "F32"), ((2, 6, 0), 2, "F32"), ((0, 6, 0), 2, "F16"),
                                             ((0, 6, 0), 4, "BF16"), ((4, 6, 0), 4, "F16"), ((0, 7, 0), 4, "F32"),
                                             ((0, 7, 0), 1, "BF16"), ((0, 6, 0), 8, "F32")])
@pytest.mark.parametrize("recon", [18, 12])
def test_interleaved_strips_bitwise_equal_single(ctx, T, tile, vb, storage, recon):
    """Strip lengths (some not dividing hx), W staged in shared memory (tile[1] = 1), the
    packed FP32 pair kernel (tile[1] = 2) and the whole-row kernel with TMA-staged W rows
    (tile[1] = 6, 7; tile[0] = vectors per CTA) == one vector per launch, bitwise."""
    dims = (12, 10, 8, 2)
    nvec = 8
    st = getattr(T, "TLS_" + storage)
    U = gauge(dims, "haar", 35)
    vecs = synth.gaussian_vectors(dims, nvec, 36, dtype=torch.complex64)
    gid = ctx.load_gauge(U, 4, dims)
    ctx.build_twolink(gid, T.TLS_F32, recon)
    ctx.tune_set(gid, nvec, st, T.TLS_ALL_T, T.TLS_KERNEL_MRHS, vb, 0, tile)
    a = vecs.clone().cuda()
    ctx.set_profiling(True)
    ctx.smear(gid, a, T.TLS_F32, nvec, 6, 1.3, storage=st, kernel=T.TLS_KERNEL_AUTO)
    assert ctx.get_profile()["kernel"] == T.TLS_KERNEL_MRHS
    ctx.set_profiling(False)
    b = vecs.clone().cuda()
    ctx.smear(gid, b, T.TLS_F32, nvec, 6, 1.3, storage=st, kernel=T.TLS_KERNEL_SINGLE)
    ctx.free_gauge(gid)
    assert torch.equal(a, b)
    if storage == "F32" and recon == 18:
        want = oracle.smear(oracle.twolink(U.numpy()), vecs.numpy().astype(np.complex128), 6, 1.3)
        assert max(per_vector_rel_l2(a.cpu().numpy().astype(np.complex128), want)) <= 2e-6 * 6


@pytest.mark.parametrize("dims,nvec,storage,wprec,recon,vb,nvg", [
    ((8, 8, 8, 3), 24, "F32", "F32", 18, 4, 0), ((16, 8, 12, 2), 24, "F32", "F32", 18, 4, 12),
    ((8, 16, 24, 2), 8, "F32", "F32", 12, 2, 0), ((12, 8, 8, 2), 12, "F32", "F32", 8, 4, 4),
    ((8, 8, 8, 2), 6, "F16", "F16", 12, 2, 0), ((16, 8, 8, 2), 8, "BF16", "BF16", 18, 4, 0),
    ((8, 4, 4, 2), 16, "F16", "F32", 18, 4, 8), ((10, 6, 4, 2), 4, "F16", "F16", 18, 2, 0),
    ((10, 6, 4, 2), 4, "F32", "F32", 18, 4, 0), ((2, 2, 2, 1), 4, "F32", "F32", 18, 4, 0),
    ((4, 4, 2, 2), 3, "F32", "F32", 18, 1, 0)])
def test_row_tma_kernel_bitwise_equal_single(ctx, T, dims, nvec, storage, wprec, recon, vb, nvg):
    """Whole-row CTAs with the five W rows staged by TMA bulk copies (tile[1] = 6, 7) == one
    vector per launch, bitwise, on every slice and on one slice; hx = 5 with a 4- or 8-byte W
    remainder plane takes the packed kernel instead (same results)."""
    U = gauge(dims, "haar", 37)
    vecs = synth.gaussian_vectors(dims, nvec, 38, dtype=torch.complex64)
    st = getattr(T, "TLS_" + storage)
    wp = getattr(T, "TLS_" + wprec)
    gid = ctx.load_gauge(U, 4, dims)
    ctx.build_twolink(gid, wp, recon)
    for t0 in (-1, dims[3] - 1):
        b = vecs.clone().cuda()
        ctx.smear(gid, b, T.TLS_F32, nvec, 7, 1.4, timeslice=t0, storage=st, kernel=T.TLS_KERNEL_SINGLE)
        # 6: the default launch bounds; 7: the next hop's records requested early;
        # 8: the row's own records staged in shared memory with the W rows;
        # pfd > 0: the rows pfd planes ahead requested into L2 (-1: about 12 MB ahead)
        for variant, pfd in ((6, 0), (7, 0), (8, 0), (6, 3), (8, 5), (6, -1), (7, -1)):
            ctx.tune_set(gid, nvec, st, t0, T.TLS_KERNEL_MRHS, vb, 0, (nvg, variant, pfd))
            a = vecs.clone().cuda()
            ctx.smear(gid, a, T.TLS_F32, nvec, 7, 1.4, timeslice=t0, storage=st, kernel=T.TLS_KERNEL_AUTO)
            assert torch.equal(a, b), (variant, pfd)
    ctx.free_gauge(gid)
    if storage == "F32" and recon == 18:  # the last slice (smeared alone) against the oracle
        want = oracle.smear(oracle.twolink(U.numpy()), vecs.numpy().astype(np.complex128), 7, 1.4)
        got = a.cpu().numpy().astype(np.complex128)
        assert max(per_vector_rel_l2(got[:, -1:], want[:, -1:])) <= 2e-6 * 7


def test_peak_flops_measures_the_fma_rates(T):
    """tls_peak_flops: positive rates, packed FP32 at least the scalar FP32 rate within the
    timing noise, and FP32 well above FP64 on this GPU (the roof of the FP64 kernels)."""
    f64 = T.tls_peak_flops(0, T.TLS_PEAK_F64)
    f32 = T.tls_peak_flops(0, T.TLS_PEAK_F32)
    f2 = T.tls_peak_flops(0, T.TLS_PEAK_F32X2)
    assert f64 > 0 and f32 > 0 and f2 > 0
    assert f2 >= 0.9 * f32
    assert f32 > 4 * f64
    with pytest.raises(T.TLSError):
        T.tls_peak_flops(0, 7)


# ------------------------------------------------------------------ one-link Gaussian smearing (Eq. 2-3)
@pytest.mark.parametrize("storage,nvec,t0,dims", [("F64", 3, -1, (6, 4, 8, 3)), ("F32", 4, 1, (8, 8, 4, 2)),
                                                  ("F32", 5, -1, (2, 6, 4, 2)), ("F16", 6, -1, (8, 4, 6, 2)),
                                                  ("BF16", 2, 0, (4, 4, 4, 1))])
def test_onelink_smear_matches_oracle(ctx, T, storage, nvec, t0, dims):
    U = gauge(dims, "haar", 41)
    vecs = synth.gaussian_vectors(dims, nvec, 42)
    N, alpha = 6, 0.09
    want = oracle.smear_onelink(U.numpy(), vecs.numpy(), N, alpha, t0=t0)
    st = getattr(T, "TLS_" + storage)
    gid = ctx.load_gauge(U, 4, dims)
    ctx.build_links(gid, T.TLS_F64 if st == T.TLS_F64 else T.TLS_F32)
    x = vecs.to(torch.complex128 if st == T.TLS_F64 else torch.complex64).cuda()
    norms = ctx.smear_onelink(gid, x, T.TLS_F64 if st == T.TLS_F64 else T.TLS_F32, nvec, N, alpha, timeslice=t0,
                              storage=st, norms=True)
    ctx.free_gauge(gid)
    got = x.cpu().numpy().astype(np.complex128)
    errs = per_vector_rel_l2(got, want)
    assert max(errs) <= tol(st, N), errs
    sl = slice(None) if t0 < 0 else slice(t0, t0 + 1)
    assert np.allclose(norms, (np.abs(got[:, sl]) ** 2).reshape(nvec, -1).sum(1), rtol=1e-12, atol=0)


def test_onelink_needs_links(ctx, T):
    dims = (4, 4, 4, 1)
    gid = ctx.load_gauge(gauge(dims, "haar", 43), 4, dims)
    x = synth.gaussian_vectors(dims, 1, 44, dtype=torch.complex64).cuda()
    with pytest.raises(T.TLSError) as e:
        ctx.smear_onelink(gid, x, T.TLS_F32, 1, 3, 0.1)
    assert e.value.status == T.TLS_ERR_NOT_BUILT
    ctx.build_links(gid, T.TLS_F32)
    with pytest.raises(T.TLSError) as e:
        ctx.smear_onelink(gid, x.to(torch.complex128), T.TLS_F64, 1, 3, 0.1, storage=T.TLS_F64)
    assert e.value.status == T.TLS_ERR_UNSUPPORTED
    ctx.free_gauge(gid)


# ------------------------------------------------------------------ many-source sink smearing (Sec. 6)
def test_sink_smear_pattern_small(ctx, T):
    """72 dense vectors on every slice, n = 30, one W: the many-source batch against the oracle."""
    dims = (8, 8, 8, 4)
    w = workloads.SINK_SMEAR
    U = gauge(dims, "near", 45, eps=0.2)
    vecs = synth.gaussian_vectors(dims, w["nvec"], 46, dtype=torch.complex64)
    want = oracle.smear(oracle.twolink(U.numpy()), vecs.numpy().astype(np.complex128), w["N"], w["sigma"])
    got, norms = _run(ctx, T, U, dims, vecs, T.TLS_F32, T.TLS_F32, 18, T.TLS_KERNEL_MRHS, w["N"], w["sigma"], -1)
    errs = per_vector_rel_l2(got, want)
    assert max(errs) <= tol(T.TLS_F32, w["N"]), max(errs)
    assert np.allclose(norms, (np.abs(got) ** 2).reshape(w["nvec"], -1).sum(1), rtol=1e-12, atol=0)


def test_sink_smear_workload_sampled(ctx, T):
    """48^3x64 with 72 dense vectors, n = 30 (the sink-smearing workload), sampled against the oracle."""
    w = workloads.SINK_SMEAR
    dims = w["dims"]
    U = gauge_dev(dims, "near", w["gauge_seed"], eps=w["eps"], nd=4)
    vecs = synth.gaussian_vectors(dims, w["nvec"], w["vec_seed"], dtype=torch.complex64, device="cuda")
    samples = ((0, 0), (37, 29), (71, 63))
    ref = {(v, t): vecs[v, t:t + 1].cpu().numpy().astype(np.complex128) for v, t in samples}
    gid = ctx.load_gauge(U, 4, dims)
    ctx.build_twolink(gid, T.TLS_F32, 18)
    ctx.smear(gid, vecs, T.TLS_F32, w["nvec"], w["N"], w["sigma"], storage=T.TLS_F32, kernel=T.TLS_KERNEL_AUTO)
    ctx.free_gauge(gid)
    for (v, t), src in ref.items():
        want = oracle.smear(oracle.twolink(U[t:t + 1].cpu().numpy()), src, w["N"], w["sigma"])
        got = vecs[v, t:t + 1].cpu().numpy().astype(np.complex128)
        assert rel_l2(got, want) <= tol(T.TLS_F32, w["N"])
    del vecs, U
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ APE-smeared links (Sec. 2)
@pytest.mark.parametrize("dims,alpha,n", [((6, 4, 8, 2), 0.45, 3), ((4, 4, 4, 1), 0.7, 1), ((8, 6, 4, 3), 0.2, 2)])
def test_ape_matches_oracle(ctx, T, dims, alpha, n):
    U = gauge(dims, "haar", 61)
    want = oracle.ape_smear(U.numpy(), alpha, n)
    gid = ctx.load_gauge(U, 4, dims)
    ctx.ape_smear(gid, alpha, n)
    got = np.zeros_like(want)
    ctx.export_gauge(gid, got)
    ctx.free_gauge(gid)
    assert np.abs(got - want).max() < 1e-12


def test_ape_then_twolink_smear(ctx, T):
    """Smeared links feed the two-link build: the whole chain against the oracle's."""
    dims = (6, 6, 4, 2)
    U = gauge(dims, "near", 62, eps=0.4)
    vecs = synth.gaussian_vectors(dims, 3, 63)
    Ua = oracle.ape_smear(U.numpy(), 0.5, 2)
    want = oracle.smear(oracle.twolink(Ua), vecs.numpy(), 7, 1.4)
    gid = ctx.load_gauge(U, 4, dims)
    ctx.ape_smear(gid, 0.5, 2)
    ctx.build_twolink(gid, T.TLS_F64, 18)
    x = vecs.clone().cuda()
    ctx.smear(gid, x, T.TLS_F64, 3, 7, 1.4, storage=T.TLS_F64, kernel=T.TLS_KERNEL_MRHS)
    ctx.free_gauge(gid)
    assert max(per_vector_rel_l2(x.cpu().numpy(), want)) <= 1e-13


def test_ape_pure_gauge_and_state(ctx, T):
    dims = (4, 6, 4, 2)
    G = synth.gauge_transform_haar(dims, 64).numpy()
    U = np.empty(G.shape[:4] + (3, 3, 3), dtype=np.complex128)
    for i, ax in enumerate((3, 2, 1)):
        U[..., i, :, :] = G @ np.conj(np.swapaxes(np.roll(G, -1, axis=ax), -1, -2))
    gid = ctx.load_gauge(torch.from_numpy(U), 3, dims)
    ctx.build_twolink(gid, T.TLS_F32, 18)
    ctx.ape_smear(gid, 0.6, 2)
    got = np.zeros_like(U)
    ctx.export_gauge(gid, got)
    assert np.abs(got - U).max() < 1e-12
    x = synth.gaussian_vectors(dims, 1, 65, dtype=torch.complex64).cuda()
    with pytest.raises(T.TLSError) as e:  # W predates the smearing
        ctx.smear(gid, x, T.TLS_F32, 1, 2, 0.5)
    assert e.value.status == T.TLS_ERR_NOT_BUILT
    with pytest.raises(T.TLSError) as e:
        ctx.ape_smear(gid, 1.5, 1)
    assert e.value.status == T.TLS_ERR_ARG
    ctx.free_gauge(gid)


def test_ape_large_lattice_sampled(ctx, T):
    """32^3 x 4: one slice of the device result against the oracle on that slice alone."""
    dims = (32, 32, 32, 4)
    U = gauge_dev(dims, "near", 66, eps=0.3, nd=4)
    gid = ctx.load_gauge(U, 4, dims)
    ctx.ape_smear(gid, 0.5, 2)
    got = torch.zeros(dims[3], dims[2], dims[1], dims[0], 3, 3, 3, dtype=torch.complex128, device="cuda")
    ctx.export_gauge(gid, got)
    ctx.free_gauge(gid)
    t = 2
    want = oracle.ape_smear(U[t:t + 1].cpu().numpy(), 0.5, 2)
    assert np.abs(got[t:t + 1].cpu().numpy() - want).max() < 1e-12


# ------------------------------------------------------------------ on-chip persistent form
@pytest.mark.parametrize("dims,nvec,storage,vb", [((8, 8, 8, 3), 5, "F32", 1), ((16, 16, 16, 2), 6, "F32", 4),
                                                  ((16, 8, 8, 2), 7, "F16", 1), ((8, 8, 8, 2), 3, "F64", 1),
                                                  ((16, 16, 16, 1), 9, "BF16", 4), ((4, 4, 4, 2), 2, "F32", 1)])
def test_persistent_onchip_bitwise_equals_l2_form(ctx, T, dims, nvec, storage, vb):
    """One CTA per block with W and the iterates in shared memory == the grid-wide persistent kernel."""
    st = getattr(T, "TLS_" + storage)
    io = T.TLS_F64 if st == T.TLS_F64 else T.TLS_F32
    dt = torch.complex128 if io == T.TLS_F64 else torch.complex64
    U = gauge(dims, "haar", 71)
    vecs = synth.gaussian_vectors(dims, nvec, 72, dtype=dt)
    gid = ctx.load_gauge(U, 4, dims)
    ctx.build_twolink(gid, T.TLS_F64 if st == T.TLS_F64 else T.TLS_F32, 18)
    b = vecs.clone().cuda()
    ctx.smear(gid, b, io, nvec, 9, 1.7, storage=st, kernel=T.TLS_KERNEL_PERSISTENT)
    ctx.tune_set(gid, nvec, st, T.TLS_ALL_T, T.TLS_KERNEL_PERSISTENT, vb, 1024 if nvec % 2 else 512, (0, 1, 0))
    a = vecs.clone().cuda()
    ctx.set_profiling(True)
    ctx.smear(gid, a, io, nvec, 9, 1.7, storage=st, kernel=T.TLS_KERNEL_AUTO)
    assert ctx.get_profile()["kernel"] == T.TLS_KERNEL_PERSISTENT
    ctx.set_profiling(False)
    ctx.free_gauge(gid)
    assert torch.equal(a, b)
    if storage == "F32":
        want = oracle.smear(oracle.twolink(U.numpy()), vecs.numpy().astype(np.complex128), 9, 1.7)
        assert max(per_vector_rel_l2(a.cpu().numpy().astype(np.complex128), want)) <= 2e-6 * 9
