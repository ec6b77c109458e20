"""tls_smear_noalloc: the smear for callers that cannot allocate device memory.

Some callers may not call cudaMalloc while they run: a latency-critical
thread (cudaFree synchronises the device), or a process whose device memory
belongs to another allocator.  This entry
point keeps all its intermediate data in a fixed static device array owned by
the library.  The test calls it through the C ABI twice in a row and checks
each result against tls_smear with the persistent kernel (the existing entry
point it mirrors), within the FP32 tolerance the other tests use.  It also
checks that the context's device memory does not grow, and that a smear too
large for the array is refused with an error.

This file is collected last on purpose (pytest orders test files by name).
"""

import numpy as np
import pytest
import torch

from helpers import per_vector_rel_l2
from paper_2301_05518_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2301_05518_gb300 import tls as t
    return t


def test_noalloc_matches_persistent_smear_twice(T):
    dims = (8, 8, 8, 4)
    N, sigma = 9, 1.8
    with T.Context(0) as ctx:
        U = synth.gauge_haar(dims, 91, nd=4)
        gid = ctx.load_gauge(U, 4, dims)
        ctx.build_twolink(gid, T.TLS_F32, T.TLS_R18)
        for call, seed in enumerate((92, 93)):
            vecs = synth.gaussian_vectors(dims, 3, seed, dtype=torch.complex64).cuda()
            ref = vecs.clone()
            ctx.smear(gid, ref, T.TLS_F32, 3, N, sigma, storage=T.TLS_F32, kernel=T.TLS_KERNEL_PERSISTENT)
            got = vecs.clone()
            torch.cuda.synchronize()
            before = ctx.bytes_in_use()
            free_before = torch.cuda.mem_get_info()[0]
            ctx.smear_noalloc(gid, got, T.TLS_F32, 3, N, sigma, storage=T.TLS_F32)
            assert ctx.bytes_in_use() == before
            if call > 0:  # warmed up: the device's free memory does not move either
                assert torch.cuda.mem_get_info()[0] == free_before
            errs = per_vector_rel_l2(got.cpu().numpy().astype(np.complex128),
                                     ref.cpu().numpy().astype(np.complex128))
            assert max(errs) <= 2e-6 * N, (call, errs)
        # one slice, FP32; then 16-bit storage with its per-site scales (FP32 scratch)
        for storage, t0, tol in ((T.TLS_F32, 1, 2e-6 * N), (T.TLS_F16, -1, 5e-3), (T.TLS_BF16, 3, 5e-3)):
            vecs = synth.gaussian_vectors(dims, 4, 96 + storage, dtype=torch.complex64).cuda()
            ref = vecs.clone()
            ctx.smear(gid, ref, T.TLS_F32, 4, N, sigma, timeslice=t0, storage=storage,
                      kernel=T.TLS_KERNEL_PERSISTENT)
            got = vecs.clone()
            ctx.smear_noalloc(gid, got, T.TLS_F32, 4, N, sigma, timeslice=t0, storage=storage)
            errs = per_vector_rel_l2(got.cpu().numpy().astype(np.complex128),
                                     ref.cpu().numpy().astype(np.complex128))
            assert max(errs) <= tol, (storage, t0, errs)
        # one slice only, FP64
        ctx.build_twolink(gid, T.TLS_F64, T.TLS_R18)
        vecs = synth.gaussian_vectors(dims, 2, 94).cuda()
        ref = vecs.clone()
        ctx.smear(gid, ref, T.TLS_F64, 2, N, sigma, timeslice=2, storage=T.TLS_F64,
                  kernel=T.TLS_KERNEL_PERSISTENT)
        got = vecs.clone()
        ctx.smear_noalloc(gid, got, T.TLS_F64, 2, N, sigma, timeslice=2, storage=T.TLS_F64)
        errs = per_vector_rel_l2(got.cpu().numpy(), ref.cpu().numpy())
        assert max(errs) <= 1e-13
        ctx.free_gauge(gid)


def test_noalloc_rejects_oversize(T):
    dims = (32, 32, 32, 8)
    with T.Context(0) as ctx:
        U = synth.gauge_haar(dims, 95, nd=4, device="cuda")
        gid = ctx.load_gauge(U, 4, dims)
        ctx.build_twolink(gid, T.TLS_F32, T.TLS_R18)
        x = torch.zeros((4,) + (dims[3], dims[2], dims[1], dims[0], 3), dtype=torch.complex64, device="cuda")
        with pytest.raises(T.TLSError) as e:
            ctx.smear_noalloc(gid, x, T.TLS_F32, 4, 5, 1.0)
        assert e.value.status == T.TLS_ERR_ARG
        host = torch.zeros((1, 4, 4, 4, 4, 3), dtype=torch.complex64)
        with pytest.raises(T.TLSError):
            ctx.smear_noalloc(gid, host, T.TLS_F32, 1, 5, 1.0)
        ctx.free_gauge(gid)
