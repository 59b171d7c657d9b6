"""CPU pin of the finite-difference method (tests/fd_check.py) on the oracle itself:
its FP64 adjoint, restricted to the rays on which each parameter is smooth, equals
the per-ray central differences of its forward (reduced differentiation workload)."""
import numpy as np

import fd_check as F
import oracle


def test_oracle_adjoint_matches_per_ray_finite_differences():
    prob = F.Problem("diff_small_64x8^3_2x48x40", seed=0, n_prims=2)
    whole = prob.oracle_grads()

    def grad_of_rays(kind, idx, rays):
        return oracle.backward(prob.sc, prob._sub(rays), prob.grad_out[rays], F.F64M)[kind][idx]

    params = prob.params(whole["g_payload"], n_payload=8, n_pose=8)
    e_pay, _, _ = F.check(prob, whole, grad_of_rays, [p for p in params if p[0] == "g_payload"], "payload", h=F.H)
    e_pose, fr, _ = F.check(prob, whole, grad_of_rays, [p for p in params if p[0] != "g_payload"], "pose",
                            h=F.H_POSE)
    assert e_pay.max() <= 1e-6
    assert e_pose.max() <= F.TOL
    # planted mistake: a gradient off by 1 % fails the bar
    bad = {k: v.copy() for k, v in whole.items()}
    kind, idx = params[-1]

    def off(kd, ix, rays):
        g = grad_of_rays(kd, ix, rays)
        return g * 1.01 if (kd, ix) == (kind, idx) else g

    e_bad, _, _ = F.check(prob, bad, off, [params[-1]], "planted 1 % error", h=F.H_POSE)
    assert e_bad.max() > F.TOL
