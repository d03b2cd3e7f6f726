"""The allocation-free solve (ot_solve_gravity_static) against the
allocating one (ot_solve_gravity).

Callers that cannot allocate device memory -- plug-ins whose host
application owns the device memory, loops that forbid allocation after
start-up -- use the static entry point; it must give the same answer as the
normal path, call after call, although every call reuses the same fixed
scratch array.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2412_15518_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-6


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def test_static_solve_matches_the_allocating_solve_twice_in_a_row():
    assert torch.cuda.is_available()
    from paper_2412_15518_gb300 import fmm
    leaves = I.uniform_leaves(1, seed=5)
    rho_a = torch.from_numpy(I.density(leaves, I.SPHERE, seed=1)).cuda()
    rho_b = torch.from_numpy(I.density(leaves, I.BINARY, seed=2)).cuda()
    tree = fmm.Tree(leaves)
    for prec, tol in ((fmm.OT_PRECISION_FP64, TOL64), (fmm.OT_PRECISION_FP32_BULK, TOL32),
                      (fmm.OT_PRECISION_FP32_WIDE, TOL32)):
        opts = fmm.make_opts(precision=prec)
        refs = [tree.solve(r, precision=prec) for r in (rho_a, rho_b)]
        refs = [(p.clone(), g.clone()) for p, g in refs]
        # two calls in a row on the same scratch, different densities
        for r, (p_ref, g_ref) in zip((rho_a, rho_b), refs):
            phi = torch.full_like(p_ref, float("nan"))
            g = torch.full_like(g_ref, float("nan"))
            fmm.ot_solve_gravity_static(leaves, r, phi, g, opts)
            torch.cuda.synchronize()
            assert rel(phi, p_ref) < tol
            assert rel(g, g_ref) < tol
    tree.close()


def test_static_solve_rejects_trees_beyond_its_limit():
    from paper_2412_15518_gb300 import fmm
    leaves = I.uniform_leaves(2)  # 73 nodes > 9
    rho = torch.ones((leaves.shape[0], 512), dtype=torch.float64, device="cuda")
    phi = torch.empty_like(rho)
    g = torch.empty((leaves.shape[0], 3, 512), dtype=torch.float64, device="cuda")
    with pytest.raises(fmm.OTError) as e:
        fmm.ot_solve_gravity_static(leaves, rho, phi, g)
    assert e.value.code == -11
    # the root leaf alone is within the limit
    root = np.array([[0, 0, 0, 0]], np.int32)
    r1 = torch.from_numpy(I.density(root, I.SPHERE, seed=3)).cuda()
    p1, g1 = torch.empty_like(r1), torch.empty((1, 3, 512), dtype=torch.float64, device="cuda")
    fmm.ot_solve_gravity_static(root, r1, p1, g1)
    tree = fmm.Tree(root)
    p2, g2 = tree.solve(r1)
    torch.cuda.synchronize()
    assert rel(p1, p2) < TOL64 and rel(g1, g2) < TOL64
    tree.close()


def test_static_solve_on_a_caller_stream_and_option_checks():
    """On a non-default stream the call is ordered on that stream: two calls
    in a row there, each read after that stream alone is synchronised.  Bad
    options are rejected as ot_solve_gravity rejects them."""
    from paper_2412_15518_gb300 import fmm
    leaves = I.uniform_leaves(1, seed=2)
    rho_a = torch.from_numpy(I.density(leaves, I.BINARY, seed=4)).cuda()
    rho_b = torch.from_numpy(I.density(leaves, I.SPHERE, seed=6)).cuda()
    tree = fmm.Tree(leaves)
    refs = [tuple(x.clone() for x in tree.solve(r)) for r in (rho_a, rho_b)]
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    for r, (p_ref, g_ref) in zip((rho_a, rho_b), refs):
        phi = torch.full_like(p_ref, float("nan"))
        g = torch.full_like(g_ref, float("nan"))
        torch.cuda.synchronize()
        fmm.ot_solve_gravity_static(leaves, r, phi, g, fmm.make_opts(), stream=side)
        side.synchronize()
        assert rel(phi, p_ref) < TOL64
        assert rel(g, g_ref) < TOL64
    phi, g = torch.empty_like(refs[0][0]), torch.empty_like(refs[0][1])
    for bad in (dict(G=float("nan")), dict(theta=0.4), dict(precision=7)):
        with pytest.raises(fmm.OTError) as e:
            fmm.ot_solve_gravity_static(leaves, rho_a, phi, g, fmm.make_opts(**bad))
        assert e.value.code == -1, bad
    tree.close()
