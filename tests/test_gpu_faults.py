"""Failure paths made on the host, with no GPU fault: an allocation the
device cannot satisfy, and checkpoint blobs that are cut short or
corrupted.  Each must come back as an error code, leave nothing allocated
and leave the library usable."""
import ctypes

import numpy as np
import pytest

import mlba_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_1504_07234_gb300.build import build
    build()
    import paper_1504_07234_gb300 as mod
    return mod


def test_oversized_batch_reports_nomem_and_leaks_nothing(M):
    """A batch whose arena exceeds the device memory: mlba_batch_create
    returns MLBA_E_NOMEM after the host set-up, frees what it took, and
    leaves no stale error behind (the next batch creates and runs)."""
    import torch
    torch.cuda.init()
    lib = M.load_library()
    free0, total = torch.cuda.mem_get_info()
    n, p = 4096, 31
    # FP64, two levels: the two Bregman buffers alone take 2 * 17 * 8 (n + p - 1)^2 bytes
    per = 2 * 17 * 8 * (n + p - 1) ** 2
    count = int(2 * total // per) + 1
    psf = np.ascontiguousarray(I.psf_gaussian(5.0, p), dtype=np.float64)
    descs = (M.ProblemDesc * count)()
    for d in descs:
        d.psf = psf.ctypes.data_as(ctypes.c_void_p)
        d.p, d.n = p, n
        d.bc, d.precond, d.transform = M.BC["rect"], M.PRECOND["bccb"], M.TRANSFORM["dct"]
        d.max_iter, d.mu, d.alpha, d.delta = 10, 10 / 255, 0.5, 1.0
        d.g, d.g_on_device = None, 0
    opts = M.make_opts(dtype="f64", levels=2, max_iter=10)
    h = ctypes.c_void_p()
    rc = lib.mlba_batch_create(descs, count, ctypes.byref(opts), ctypes.byref(h))
    assert rc == -2, rc                                  # MLBA_E_NOMEM
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 64 << 20, (free0, free1)  # nothing kept
    # the library and the context stay usable
    pr = I.config(2, n=64)
    ctx = M.Context(pr.psf, pr.n, pr.bc, pr.precond, dtype="f32", mu=pr.mu, levels=2,
                    max_iter=3, stop=False, transform="dct")
    ctx.set_data(pr.g, pr.delta)
    ctx.run(3)
    st = ctx.stats()
    assert st["iter"] == 3 and st["status"] == 0
    ctx.close()


def test_truncated_or_corrupted_checkpoint_is_refused(M):
    """mlba_set_state refuses a blob one byte short, one with a damaged
    header and one whose iteration count is past the budget, changes nothing
    when it refuses, and still accepts the intact blob afterwards."""
    pr = I.config(2, n=64)
    a = M.Context(pr.psf, pr.n, pr.bc, pr.precond, dtype="f64", mu=pr.mu, levels=2,
                  max_iter=8, stop=False, transform="dct")
    a.set_data(pr.g, pr.delta)
    a.iterate(4)
    blob = a.get_state()
    f4 = a.result()
    a.iterate(2)
    st6, f6 = a.stats(), a.result()
    bad_magic = bytearray(blob)
    bad_magic[0] ^= 0xFF
    bad_iter = bytearray(blob)
    bad_iter[4 * 15:4 * 16] = np.int32(1000).tobytes()   # StateHeader.iter: past max_iter
    for bad in (blob[:-1], bytes(bad_magic), bytes(bad_iter)):
        with pytest.raises(M.MlbaError):
            a.set_state(bad)
        assert a.stats() == st6
        np.testing.assert_array_equal(a.result(), f6)
    a.set_state(blob)
    np.testing.assert_array_equal(a.result(), f4)
    assert a.stats()["iter"] == 4
    a.close()
