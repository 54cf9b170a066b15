"""Batched solves over concurrent streams, eager and replayed from one captured CUDA graph,
must reproduce the single-pencil solves bit for bit (same kernels, same order)."""
import numpy as np
import pytest

import gep_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gep():
    import torch
    assert torch.cuda.is_available()
    from paper_1504_06443_gb300 import build
    build.build()
    import paper_1504_06443_gb300 as g
    g.load()
    return g


def dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _batch(seed0, orders):
    As, Bs = [], []
    for i, M in enumerate(orders):
        tb = gi.tight_binding(M, seed=seed0 + i)
        As.append(dev(tb["A"]))
        Bs.append(dev(tb["B"]))
    return As, Bs


def test_batched_eager_and_graph_match_single(gep):
    import torch
    orders = gi.batch_orders(12, seed=77, lo=64, hi=384)
    As, Bs = _batch(1000, orders)
    precisions = ["fp64_emulated" if M >= 256 else "fp64" for M in orders]
    bs = gep.BatchedSolver(As, Bs, nstreams=4, precisions=precisions, batch_small=0)
    bs.run()
    torch.cuda.synchronize()
    assert bs.info() == 0
    for (w, Y), A, B, p in zip(bs.results(), As, Bs, precisions):
        w1, Y1, info = gep.solve(A, B, precision=p)
        assert info == 0
        assert torch.equal(w, w1) and torch.equal(Y, Y1)
    # capture once, then replay on new inputs written into the same buffers
    bs.capture()
    As2, Bs2 = _batch(2000, orders)
    for a, a2, b, b2 in zip(As, As2, Bs, Bs2):
        a.copy_(a2)
        b.copy_(b2)
    bs.replay()
    torch.cuda.synchronize()
    assert bs.info() == 0
    for (w, Y), A, B, p in zip(bs.results(), As2, Bs2, precisions):
        w1, Y1, _ = gep.solve(A, B, precision=p)
        assert torch.equal(w, w1) and torch.equal(Y, Y1)


def test_autotuner_picks_an_engine_per_bucket(gep):
    orders = [64, 300]
    As, Bs = _batch(3000, orders)
    tuner = gep.Autotuner()
    choice = tuner.tune(As, Bs, reps=1)
    assert set(choice) == {128, 512}
    assert all(v in ("fp64", "fp64_emulated") for v in choice.values())


def _two_norm(A):
    return float(np.max(np.abs(np.linalg.eigvalsh(A))))


@pytest.fixture(scope="module")
def batch_vs_oracle(oracle_lib):
    """24 tight-binding pencils shaped like the batched workload (orders log-uniform in
    [64, 2048], multiples of 4, the largest order 2048 included), each with the oracle's
    full FP64 solve and its 2-norm."""
    orders = gi.batch_orders(24, seed=1234)
    orders[int(np.argmax(orders))] = 2048
    pencils = []
    for i, M in enumerate(orders):
        tb = gi.tight_binding(M, seed=5000 + i)
        w_ref, Y_ref, info = oracle_lib.gep_solve(tb["A"], tb["B"])
        assert info == 0
        pencils.append(dict(A=tb["A"], B=tb["B"], w=w_ref, Y=Y_ref, nA=_two_norm(tb["A"])))
    return orders, pencils


def _check_against_oracle(results, pencils, what):
    for i, ((w, Y), p) in enumerate(zip(results, pencils)):
        A, B, nA = p["A"], p["B"], p["nA"]
        M = A.shape[0]
        wh, Yh = w.cpu().numpy(), Y.cpu().numpy()
        dl = float(np.max(np.abs(wh - p["w"])))
        assert dl <= 1e-11 * nA, (what, i, M, dl)
        res = np.linalg.norm(A @ Yh - (B @ Yh) * wh[None, :]) / (np.linalg.norm(A) * M)
        assert res <= 1e-13, (what, i, M, res)
        orth = float(np.max(np.abs(Yh.T @ B @ Yh - np.eye(M))))
        assert orth <= 1e-12, (what, i, M, orth)
        # isolated eigenpairs compare element by element (both sides apply the sign convention)
        gaps = np.minimum(np.diff(p["w"], prepend=-np.inf), np.diff(p["w"], append=np.inf))
        iso = gaps > 1e-6 * nA
        if iso.any():
            assert float(np.max(np.abs(Yh[:, iso] - p["Y"][:, iso]))) <= 1e-8, (what, i, M)


@pytest.mark.parametrize("precision", ["fp64_emulated", "mixed_refined"])
def test_batched_workload_shapes_vs_oracle(gep, batch_vs_oracle, precision):
    """Every pencil of a batch spanning the batched workload's order range, solved on
    concurrent streams (eager, then replayed from one captured CUDA graph into zeroed output
    buffers), matches the FP64 oracle at the FP64 tolerances: eigenvalues, residual,
    B-orthonormality, and isolated eigenvectors element by element."""
    import torch
    orders, pencils = batch_vs_oracle
    As = [dev(p["A"]) for p in pencils]
    Bs = [dev(p["B"]) for p in pencils]
    bs = gep.BatchedSolver(As, Bs, nstreams=8, precision=precision, batch_small=0)
    bs.run()
    torch.cuda.synchronize()
    assert bs.info() == 0
    _check_against_oracle(bs.results(), pencils, "eager")
    bs.capture()
    for w, Yt in zip(bs.w, bs.Yt):
        w.zero_()
        Yt.zero_()
    bs.replay()
    torch.cuda.synchronize()
    assert bs.info() == 0
    _check_against_oracle(bs.results(), pencils, "graph")


def test_batched_small_pencils_one_cta_vs_oracle(gep, oracle_lib):
    """Pencils of order <= 128 solved whole by one CTA each in one persistent launch (the
    rest of the batch on the streams), eager and replayed from a captured graph, against the
    oracle at the FP64 tolerances."""
    import torch
    orders = [64, 72, 128, 100, 96, 256, 68, 120, 88, 340, 64, 112]
    pencils = []
    for i, M in enumerate(orders):
        tb = gi.tight_binding(M, seed=7000 + i)
        w_ref, Y_ref, info = oracle_lib.gep_solve(tb["A"], tb["B"])
        assert info == 0
        pencils.append(dict(A=tb["A"], B=tb["B"], w=w_ref, Y=Y_ref, nA=_two_norm(tb["A"])))
    As = [dev(p["A"]) for p in pencils]
    Bs = [dev(p["B"]) for p in pencils]
    bs = gep.BatchedSolver(As, Bs, nstreams=4, precision="fp64_emulated", batch_small=128)
    bs.run()
    torch.cuda.synchronize()
    assert bs.info() == 0
    _check_against_oracle(bs.results(), pencils, "eager")
    bs.capture()
    for w, Yt in zip(bs.w, bs.Yt):
        w.zero_()
        Yt.zero_()
    bs.replay()
    torch.cuda.synchronize()
    assert bs.info() == 0
    _check_against_oracle(bs.results(), pencils, "graph")


def test_batched_small_pencil_status(gep):
    """A small pencil whose B is not positive definite reports its first bad leading minor
    through the batched status, like the staged workflow; a NaN reports GEP_ERR_NONFINITE."""
    import torch
    good = gi.tight_binding(64, seed=1)
    Bbad = np.array(good["B"])
    Bbad[10, 10] = -1.0
    As = [dev(good["A"]), dev(good["A"])]
    Bs = [dev(good["B"]), dev(Bbad)]
    bs = gep.BatchedSolver(As, Bs, nstreams=1, batch_small=128)
    bs.run()
    torch.cuda.synchronize()
    assert bs.info() > 0
    An = np.array(good["A"])
    An[5, 3] = An[3, 5] = np.nan
    bs2 = gep.BatchedSolver([dev(good["A"]), dev(An)], [dev(good["B"]), dev(good["B"])], nstreams=1, batch_small=128)
    bs2.run()
    torch.cuda.synchronize()
    assert bs2.info() == gep.ERR_NONFINITE


def test_autotuner_small_choice(gep):
    orders = [64, 80, 96, 128]
    As, Bs = _batch(3100, orders)
    As2, Bs2 = _batch(3200, [300, 520])
    tuner = gep.Autotuner()
    tuner.tune(As[:1] + As2, Bs[:1] + Bs2, reps=1)
    assert tuner.tune_small(As + As2, Bs + Bs2) in (0, 128)


def test_batched_per_pencil_routes_vs_oracle(gep, batch_vs_oracle):
    """Per-pencil options (gep_solve_batched_opts): the larger pencils on the 2-stage route,
    the others 1-stage, one-CTA route for order <= 128; eager and replayed from a graph,
    every pencil against the oracle at the FP64 tolerances."""
    import torch
    orders, pencils = batch_vs_oracle
    As = [dev(p["A"]) for p in pencils]
    Bs = [dev(p["B"]) for p in pencils]
    seps = ["2stage" if M >= 256 else "1stage" for M in orders]
    bs = gep.BatchedSolver(As, Bs, nstreams=6, precision="fp64_emulated", seps=seps, batch_small=128)
    bs.run()
    torch.cuda.synchronize()
    assert bs.info() == 0
    _check_against_oracle(bs.results(), pencils, "eager")
    bs.capture()
    assert 0 < bs.graph_kernels <= bs.eager_kernels + 64
    for w, Yt in zip(bs.w, bs.Yt):
        w.zero_()
        Yt.zero_()
    bs.replay()
    torch.cuda.synchronize()
    assert bs.info() == 0
    _check_against_oracle(bs.results(), pencils, "graph")


def test_batched_legacy_entry_matches_per_pencil_options(gep):
    """gep_solve_batched (one options struct plus a precision per pencil) and
    gep_solve_batched_opts with the equivalent per-pencil structs give the same bits."""
    import ctypes
    import torch
    orders = [300, 64, 520, 140, 96]
    As, Bs = _batch(4100, orders)
    precs = ["fp64_emulated" if M >= 256 else "fp64" for M in orders]
    bs = gep.BatchedSolver(As, Bs, nstreams=3, precisions=precs, batch_small=100)
    bs.run()
    torch.cuda.synchronize()
    ref = [(w.clone(), Yt.clone()) for w, Yt in zip(bs.w, bs.Yt)]
    n = len(orders)
    o = gep.make_options(precision="fp64_emulated", batch_small=100)
    prec = (ctypes.c_int * n)(*[gep._PRECS[p] for p in precs])
    for w, Yt in zip(bs.w, bs.Yt):
        w.zero_()
        Yt.zero_()
    rc = bs.h.lib.gep_solve_batched(bs.h.h, n, bs._M, bs._A, bs._B, bs._w, bs._Y, ctypes.byref(o), prec, 3)
    assert rc == 0
    torch.cuda.synchronize()
    assert bs.info() == 0
    for (w0, Y0), w, Yt in zip(ref, bs.w, bs.Yt):
        assert torch.equal(w0, w) and torch.equal(Y0, Yt)


def test_batched_capture_refuses_oversized_graph(gep):
    """A batch whose eager run launches more kernels than the graph limit is not captured
    (the solver raises before recording anything) and still runs eagerly."""
    import torch
    As, Bs = _batch(4200, [200, 160])
    bs = gep.BatchedSolver(As, Bs, nstreams=2, batch_small=0)
    bs.GRAPH_KERNEL_LIMIT = 10
    with pytest.raises(ValueError):
        bs.capture()
    assert bs.graph is None and bs.eager_kernels > 10
    bs.run()
    torch.cuda.synchronize()
    assert bs.info() == 0
