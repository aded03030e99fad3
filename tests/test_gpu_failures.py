"""Failure detection without a GPU fault: every failure here is made on the host (a test
hook, an invalid input, an iteration budget) and must come back as a status code with
the context still usable. Nothing here traps, hangs or faults the device: the walk-stack
limit only makes the bounded walk stop early, and the allocation failure is injected in
the library's own allocation helper before cudaMalloc is called."""
import numpy as np
import pytest

import synth
from gpu_util import build_ctx, evaluate

pytestmark = pytest.mark.gpu

EINVAL, ENOMEM, ENOTBUILT, ETIMEOUT, ENOCONV = 1, 2, 4, 5, 6


def _tensors(w):
    import torch
    dev = torch.device("cuda:0")
    return (torch.as_tensor(np.ascontiguousarray(w.rho, np.float32), device=dev),
            torch.as_tensor(np.ascontiguousarray(w.td, np.float32), device=dev))


def test_fixed_point_out_of_iterations_reports_noconv():
    import torch

    import paper_2204_09072_gb300 as tr
    w = synth.with_gas(synth.turbulent_cloud(32), seed=7)  # converges in a few iterations
    ctx, t = build_ctx(w)
    tg = torch.as_tensor(w.tgas, device="cuda:0")
    td = torch.full((w.n_leaves,), 5.0, dtype=torch.float32, device="cuda:0")  # far from equilibrium
    with pytest.raises(tr.TreeRayError) as e:
        ctx.fixed_point(tg, td, max_iter=1, tol=1e-12, unroll=0)
    assert e.value.code == ENOCONV
    td.fill_(5.0)
    assert ctx.fixed_point(tg, td, max_iter=1, tol=1e-12, unroll=1, raise_on_noconv=False) == -1
    ctx.check()
    # the context stays usable: the plain solve converges afterwards
    assert ctx.fixed_point(tg, td, max_iter=200, tol=1e-4) > 0
    ctx.close()


def test_walk_stack_overflow_is_reported_and_recovers():
    import paper_2204_09072_gb300 as tr
    w = synth.random_uniform(32, seed=32, thick_frac=0.0, n_stars=1)
    ctx, _ = build_ctx(w)
    J0, F0 = evaluate(ctx)
    ctx.set_walk_stack_limit(4)  # far below what a 32^3 walk needs
    import torch
    n = w.n_leaves
    J = torch.empty(n, dtype=torch.float32, device="cuda:0")
    F = torch.empty(3 * n, dtype=torch.float64, device="cuda:0")
    ctx.evaluate(J, F)
    with pytest.raises(tr.TreeRayError) as e:
        ctx.check()
    assert e.value.code == ETIMEOUT and "stack" in str(e.value)
    ctx.walk_stats()  # the walk-only kernel has the same bounded stack
    with pytest.raises(tr.TreeRayError) as e:
        ctx.check()
    assert e.value.code == ETIMEOUT
    ctx.set_walk_stack_limit(0)
    J1, F1 = evaluate(ctx)  # checks and finds nothing
    # the deposits' shared-memory atomics may add in another order: FP32 rounding only
    assert np.allclose(J1, J0, rtol=1e-6, atol=0) and np.allclose(F1, F0, rtol=1e-5, atol=1e-6 * np.abs(F0).max())
    ctx.close()


def test_injected_allocation_failure_leaves_context_usable():
    import paper_2204_09072_gb300 as tr
    w = synth.random_uniform(8, seed=33, thick_frac=0.2, n_stars=2)
    rho, td = _tensors(w)
    ref, _ = build_ctx(w)
    J0, F0 = evaluate(ref)
    ref.close()
    failed = 0
    for k in range(1, 80):
        ctx = tr.Context(w.params)
        ctx.inject_alloc_failure(k)
        try:
            ctx.build(w.box_cm, rho, td, n=w.uniform_n, star_pos=w.star_pos, star_lum=w.star_lum)
        except tr.TreeRayError as e:
            assert e.code == ENOMEM, (k, e)
            failed += 1
            import torch
            J = torch.empty(w.n_leaves, dtype=torch.float32, device="cuda:0")
            F = torch.empty(3 * w.n_leaves, dtype=torch.float64, device="cuda:0")
            with pytest.raises(tr.TreeRayError) as e2:
                ctx.evaluate(J, F)
            assert e2.value.code == ENOTBUILT
            if k % 7 == 1:  # a later build on the same context succeeds and gives the same result
                ctx.build(w.box_cm, rho, td, n=w.uniform_n, star_pos=w.star_pos, star_lum=w.star_lum)
                J1, F1 = evaluate(ctx)
                assert np.allclose(J1, J0, rtol=1e-6, atol=0)
            ctx.close()
            continue
        ctx.close()
        break
    assert failed >= 15, failed  # every allocation of a build was made to fail once


def test_invalid_inputs_are_rejected():
    import torch

    import paper_2204_09072_gb300 as tr
    w = synth.random_uniform(8, seed=34, thick_frac=0.1, n_stars=1)
    ctx = tr.Context(w.params)
    dev = torch.device("cuda:0")
    good_rho, good_td = _tensors(w)
    bad = [("nan rho", good_rho.clone().index_fill_(0, torch.tensor([5], device=dev), float("nan")), good_td),
           ("negative rho", good_rho.clone().index_fill_(0, torch.tensor([9], device=dev), -1e-20), good_td),
           ("inf T_d", good_rho, good_td.clone().index_fill_(0, torch.tensor([3], device=dev), float("inf"))),
           ("negative T_d", good_rho, good_td.clone().index_fill_(0, torch.tensor([0], device=dev), -5.0))]
    for name, r, t in bad:
        with pytest.raises(tr.TreeRayError) as e:
            ctx.build(w.box_cm, r, t, n=w.uniform_n, star_pos=w.star_pos, star_lum=w.star_lum)
        assert e.value.code == EINVAL, name
    sp = w.star_pos.copy()
    sp[0, 1] = np.nan
    with pytest.raises(tr.TreeRayError) as e:
        ctx.build(w.box_cm, good_rho, good_td, n=w.uniform_n, star_pos=sp, star_lum=w.star_lum)
    assert e.value.code == EINVAL
    with pytest.raises(tr.TreeRayError) as e:
        ctx.build(w.box_cm, good_rho, good_td, n=w.uniform_n, star_pos=w.star_pos, star_lum=-w.star_lum)
    assert e.value.code == EINVAL
    # valid inputs on the same context build and evaluate cleanly
    ctx.build(w.box_cm, good_rho, good_td, n=w.uniform_n, star_pos=w.star_pos, star_lum=w.star_lum)
    J, F = evaluate(ctx)
    assert np.isfinite(J).all() and (J > 0).all()
    # a non-finite gas temperature in the dust balance is reported by treeray_check
    tg = torch.full((w.n_leaves,), 20.0, dtype=torch.float32, device=dev)
    tg[7] = float("nan")
    Jt = torch.as_tensor(J.astype(np.float32), device=dev)
    Td = torch.empty(w.n_leaves, dtype=torch.float32, device=dev)
    ctx.dust_temperature(tg, Jt, Td)
    with pytest.raises(tr.TreeRayError) as e:
        ctx.check()
    assert e.value.code == EINVAL and "non-finite" in str(e.value)
    ctx.check()  # the record was cleared
    ctx.close()
