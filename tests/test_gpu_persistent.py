"""The persistent schedule: the k steps of a batch as one cooperative launch
that walks the stages of a step with grid barriers in between, against the
captured-graph schedule that launches every stage separately.

Both run the same stage bodies on the same items in the same order of
reductions, so the iterates, stop iterations and statistics are compared for
equality.  The barrier waits are bounded: with a wait limit of 0 every CTA
that is not the last to arrive gives up at once, and every problem of the
batch must report MLBA_E_TIMEOUT (the launch returns; nothing hangs).
"""
import numpy as np
import pytest

import mlba_inputs as I
from test_gpu_mlba import small

pytestmark = pytest.mark.gpu

E_TIMEOUT = -4
E_UNSUPPORTED = -7


@pytest.fixture(scope="module")
def M():
    from paper_1504_07234_gb300.build import build
    build()
    import paper_1504_07234_gb300 as mod
    return mod


def mixed_problems(levels):
    """Sizes, PSFs, BCs and preconditioners of one mixed batch; the DFT and
    DCT preconditioners with fixed and nonstationary alpha, none, and the
    antireflective BC (reblurring), with budgets that stop some problems
    early."""
    probs = [small("rect", "bccb", n=40, transform="dft", iters=9, levels=levels),
             small("reflective", "tikh_ns", n=48, psf=I.psf_disk(3), transform="dct", iters=9,
                   seed=3, levels=levels),
             small("periodic", "tikh_ns", n=36, psf=I.psf_motion(5, 0.2), iters=9, seed=4,
                   levels=levels),
             small("zero", "tikh", n=70, iters=9, alpha=0.05, seed=6, levels=levels),
             small("rect", "none", n=32, iters=9, seed=7, levels=levels),
             small("antireflective", "none", n=45, psf=I.psf_gaussian(1.2, 7), alpha=1.0,
                   iters=9, seed=8, levels=levels),
             small("rect", "bccb", n=130, psf=I.psf_gaussian(1.2, 7), transform="dct", iters=9,
                   seed=5, levels=levels)]
    return [dict(psf=p.psf, g=p.g, delta=p.delta, bc=p.bc, precond=p.precond, mu=p.mu,
                 alpha=p.alpha, transform=p.transform, max_iter=3 if i == 1 else p.max_iter)
            for i, p in enumerate(probs)]


def run(M, descs, chunks, **kw):
    b = M.Batch(descs, **kw)
    for k in chunks:
        b.iterate(k)
    out = ([b.result(i) for i in range(len(descs))], [b.stats(i) for i in range(len(descs))])
    b.close()
    return out


@pytest.mark.parametrize("zs", ["f32", "bf16"])
@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("stop", [True, False])
def test_persistent_equals_graph_schedule(M, zs, levels, stop):
    descs = mixed_problems(levels)
    kw = dict(dtype="f32", z_store=zs, levels=levels, stop=stop, max_iter=9, rect_ns_hybrid=True,
              frame_shape=0)
    chunks = (1, 3, 2, 4)
    fg, sg = run(M, descs, chunks, two_group=False, **kw)
    fp, sp = run(M, descs, chunks, persistent=True, **kw)
    for i in range(len(descs)):
        assert sp[i]["status"] == 0, (i, sp[i])
        assert np.array_equal(fg[i], fp[i]), (i, float(np.abs(fg[i] - fp[i]).max()))
        assert sg[i] == sp[i], (i, sg[i], sp[i])
    assert sp[1]["iter"] == 3 and sp[1]["stopped"] == 1


def test_persistent_balanced_equals_graph_schedule(M):
    descs = mixed_problems(2)
    kw = dict(dtype="f32", levels=2, stop=False, max_iter=9, rect_ns_hybrid=True,
              formulation="balanced", frame_shape=0)
    fg, sg = run(M, descs, (2, 5), two_group=False, **kw)
    fp, sp = run(M, descs, (2, 5), persistent=True, **kw)
    for i in range(len(descs)):
        assert np.array_equal(fg[i], fp[i]), i
        assert sg[i] == sp[i], i


def test_persistent_past_the_discrepancy_point(M):
    """4-NS problems run past their discrepancy points (stop = 0), where
    alpha_n is kept and the forward column pass weights and inverts itself:
    the persistent launch equals the graphs there too."""
    probs = [small("periodic", "tikh_ns", n=48, psf=I.psf_motion(7, 0.9), alpha=0.05, iters=16,
                   nu=0.05, seed=s, levels=2) for s in (1, 2)]
    probs.append(small("reflective", "tikh_ns", n=48, psf=I.psf_disk(3), alpha=0.05, iters=16,
                       nu=0.05, transform="dct", levels=2))
    descs = [dict(psf=p.psf, g=p.g, delta=p.delta, bc=p.bc, precond=p.precond, mu=p.mu,
                  alpha=p.alpha, transform=p.transform) for p in probs]
    kw = dict(dtype="f32", levels=2, stop=False, max_iter=16, frame_shape=0)
    fg, sg = run(M, descs, (5, 12), two_group=False, **kw)
    fp, sp = run(M, descs, (5, 12), persistent=True, **kw)
    assert all(0 <= s["stop_iter"] < 16 for s in sg), sg
    for i in range(len(descs)):
        assert np.array_equal(fg[i], fp[i]), i
        assert sg[i] == sp[i], i


def test_persistent_single_problem_matches_graph(M):
    """One problem (the Context entry points) through the persistent launch."""
    p = small("reflective", "tikh_ns", n=100, psf=I.psf_disk(3), transform="dct", iters=8,
              levels=2)
    out = []
    for pers in (False, True):
        ctx = M.Context(p.psf, p.n, p.bc, p.precond, dtype="f32", mu=p.mu, alpha=p.alpha,
                        levels=2, max_iter=8, stop=False, transform="dct", frame_shape=0,
                        persistent=pers)
        ctx.set_data(p.g, p.delta)
        st = ctx.run(8)
        out.append((ctx.result(), st, ctx.history()))
        ctx.close()
    (f0, s0, h0), (f1, s1, h1) = out
    assert np.array_equal(f0, f1)
    assert s0 == s1
    for a, b in zip(h0, h1):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_persistent_barrier_timeout_reports_status(M):
    """wait_s = 0: the first grid barrier gives up, the launch returns and every
    problem stops with MLBA_E_TIMEOUT; the context stays usable."""
    descs = mixed_problems(2)
    b = M.Batch(descs, dtype="f32", levels=2, stop=False, max_iter=9, rect_ns_hybrid=True,
                persistent=True, wait_s=0.0)
    b.iterate(3)
    assert b.active() == 0
    for i in range(len(descs)):
        st = b.stats(i)
        assert st["status"] == E_TIMEOUT and st["stopped"] == 1, (i, st)
    b.close()
    # a later batch on the same device runs normally
    fg, sg = run(M, descs, (2,), dtype="f32", levels=2, stop=False, max_iter=9,
                 rect_ns_hybrid=True, persistent=True)
    assert all(s["status"] == 0 and s["iter"] == 2 for s in sg)


@pytest.mark.parametrize("kw,desc_kw", [
    (dict(dtype="f64"), {}),
    (dict(levels=3), {}),
    (dict(blur_path="fft"), {}),
    ({}, dict(bc="zero", precond="krylov", transform="dft")),
    ({}, dict(bc="antireflective", precond="bccb", transform="ar")),
])
def test_persistent_unsupported_configurations(M, kw, desc_kw):
    p = small("periodic", "tikh", n=32, iters=3)
    d = dict(psf=I.psf_gaussian(1.0, 5), g=p.g, delta=p.delta, bc="periodic", precond="tikh",
             alpha=0.1, transform="dft")
    d.update(desc_kw)
    with pytest.raises(M.MlbaError) as e:
        M.Batch([d], persistent=True, **kw)
    assert e.value.code == E_UNSUPPORTED
