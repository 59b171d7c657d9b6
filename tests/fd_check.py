"""Finite-difference check of gradients on the differentiation workload (Sec. 3.2.2).

The loss is the photometric L2 term (Sec. 3.3, lambda = 1) over a set S of rays:
L = (1/|S|) sum_{p in S} sum_rgb (I_p - target_p)^2. S is every ray of the workload's
cameras that passes near one of a few chosen primitives (FP64 depth min_t |y(t)|_inf
<= NEAR_DEPTH), so a parameter theta of primitive k changes only the rays of S near
k, and its central difference is a sum of per-ray differences rendered by the FP64
oracle (definition membership) on those rays alone.

The image is piecewise smooth in the parameters (Sec. 3.2.2's quadrature): a sample
crossing a box face switches a primitive on or off at that sample, a sample crossing
a voxel cell boundary changes the slope of the trilinear field, and the saturation
clamp moves. With tens of thousands of rays through a primitive, a step of h = 1e-3
puts such a point inside [theta - h, theta + h] on most rays, and the central
difference of the whole loss then measures the jumps, not the derivative. The check
therefore classifies each ray, per parameter: smooth when its number of (sample,
primitive) evaluations is the same at theta, theta +- h and theta +- h/2 and its
differences with steps h and h/2 agree to 1e-4 (relative, with a floor of 1e-3 of the
largest per-ray difference of that parameter); the others straddle a kink and are
counted. The gradient under test is computed with the loss restricted to the smooth
rays (the adjoint run with the loss gradient zeroed elsewhere) and compared with the
sum of their differences at h = 1e-3.

One more kink lies within rounding of theta itself: the saturation clamp (Sec. 3.2.2)
switches to the neighbouring sample when the opacity accumulated before the clamped
sample S comes within rounding of 1. The image is continuous there but its gradient
is not, and a kernel that accumulates in FP32 (an error of about 1e-6 in T) may clamp
at S - 1 or S + 1 where the FP64 oracle clamps at S. Rays whose FP64 clamp weight
beta = (1 - T_{S-1}) / a_S lies within SAT_BAND of 0 or 1 are therefore counted apart
(measured: 30 of 19458 clamped rays near one primitive of the full workload; one of
them, at beta = 4e-5, moved a quaternion entry's FP32 gradient by 0.9 %). For the same
reason a pose entry of primitive k leaves out the rays with a sample (up to the ray's
last one) within KINK_BAND of a voxel cell boundary of k (voxel units: the slope of the
trilinear field jumps there, Sec. 3.1.2) or of a face of k (local units): the kernel
places its samples in FP32 (sample time and voxel coordinate, an error up to about
1e-4 voxel units) and may take the other side. Both sets come from the FP64 geometry
(rotations through scipy) and the FP64 oracle's render at theta.

Parameters: 32 payload entries whose oracle gradient exceeds 1e-3 of the largest and
32 pose entries (t, q, s) of the chosen primitives. The step is the FP32 difference
actually made (theta +- h rounded to FP32). Error (C9 reading): |g - g_fd| /
max(|g_fd|, 1e-3 max|G|, FP32_FLOOR sum_r |g_fd,r|), G the gradient tensor of the
whole loss that the entry belongs to, g_fd,r the per-ray differences. The third term
is the conditioning of the sum: a kernel that places its samples in FP32 (about 5e-5
voxel units from the FP64 positions) gives each ray's gradient a small relative error,
and where the rays' contributions cancel (sum_r |g_fd,r| up to ~1000 |g_fd| for some
quaternion entries of the full workload) that error, not a wrong derivative, sets
|g - g_fd|. FP32_FLOOR = TOL * 3e-5 admits a per-ray error of 3e-5 of the rays'
summed magnitude (measured on the GPU: at most 1.8e-5); the plain C9 error, without
this term, is printed beside it.

Steps. The image is exactly piecewise linear in a payload entry, so payload entries
take the specified h = 1e-3. A pose step of 1e-3 moves every sample of ~30000 rays by
7-14 % of a voxel cell, so nearly every ray holds an undetected slope change and the
sum of their differences misses the derivative by up to ~16 % (measured with the
oracle's own adjoint, which converges to the differences as h shrinks); pose entries
are therefore held to the bar at H_POSE = 1e-6 (0.2 % of rays then straddle a kink
and are left out), and their h = 1e-3 errors are reported.
"""
from __future__ import annotations

import numpy as np

import oracle
import synthetic
from helpers import rays_from
from parity_rules import local_lines, pair_depth

F64M = oracle.MODE_PRUNED | oracle.MEMBER_F64
NEAR_DEPTH = 1.2
H = 1e-3
H_POSE = 1e-6
TOL = 1e-3
SMOOTH_TOL = 1e-4
SAT_BAND = 1e-3
KINK_BAND = 2e-4
FP32_FLOOR = 0.03  # x sum_r |g_fd,r| (a per-ray error of 3e-5 at TOL = 1e-3)
KEYS = {"g_payload": "payload", "g_t": "t", "g_q": "q", "g_s": "s"}


def choose_primitives(sc, rays, n_pick, seed):
    """Primitives whose centre is in front of camera 0 and on the near side of the shell."""
    cam = rays.cameras[0]
    rel = sc.t.astype(np.float64) - cam.eye[None]
    z = rel @ cam.c2w[:, 2]
    x = rel @ cam.c2w[:, 0] / np.maximum(z, 1e-9) * cam.focal + cam.width / 2
    y = rel @ cam.c2w[:, 1] / np.maximum(z, 1e-9) * cam.focal + cam.height / 2
    ok = (z > 0) & (z < np.linalg.norm(cam.eye) - 0.3) & (x > 8) & (x < cam.width - 8) & (y > 8) & \
        (y < cam.height - 8)
    cand = np.flatnonzero(ok)
    return np.sort(np.random.default_rng(seed).choice(cand, n_pick, replace=False))


class Problem:
    def __init__(self, cfg="diff_512x32^3_4x512x512", seed=0, n_prims=4):
        self.sc, self.rays, extra = synthetic.make_config(cfg, seed)
        self.target = extra["target"].reshape(-1, 3).astype(np.float64)
        self.picked = choose_primitives(self.sc, self.rays, n_prims, seed + 11)
        n = self.rays.n
        self._ol, self._dl, self.S_k = {}, {}, {}
        for k in self.picked:
            ol, dl = local_lines(self.sc, self.rays.o, self.rays.d, np.arange(n), np.full(n, int(k)))
            near = np.flatnonzero(pair_depth(ol, dl, self.rays.t_near, self.rays.t_far) <= NEAR_DEPTH)
            self.S_k[int(k)] = near
            self._ol[int(k)], self._dl[int(k)] = ol[near], dl[near]
        self.S = np.unique(np.concatenate(list(self.S_k.values())))
        self._n0 = {}  # per (kind, index): evaluations and clamp flags of each changed ray at theta
        img = oracle.render(self.sc, self._sub(self.S), F64M)["rgba"]
        self.grad_out = np.zeros((n, 4), np.float64)
        self.grad_out[self.S, :3] = 2.0 * (img[:, :3] - self.target[self.S]) / self.S.size

    def _sub(self, idx):
        r = self.rays
        return rays_from(r.o[idx], r.d[idx], r.t_near, r.t_far, r.dt)

    def oracle_grads(self, rays_idx=None):
        """The oracle's FP64 adjoint of L restricted to rays_idx (default S)."""
        idx = self.S if rays_idx is None else rays_idx
        return oracle.backward(self.sc, self._sub(idx), self.grad_out[idx], F64M)

    def params(self, g_payload_ref, seed=3, n_payload=32, n_pose=32):
        rng = np.random.default_rng(seed)
        gp = np.abs(g_payload_ref[self.picked])
        big = np.argwhere(gp > 1e-3 * gp.max())
        pick = big[rng.choice(len(big), n_payload, replace=False)]
        out = [("g_payload", (int(self.picked[p[0]]),) + tuple(int(x) for x in p[1:])) for p in pick]
        pose = [(key, (int(k), j)) for k in self.picked for key, m in (("g_t", 3), ("g_q", 4), ("g_s", 3))
                for j in range(m)]
        for i in rng.choice(len(pose), n_pose, replace=False):
            out.append(pose[i])
        return out

    def rays_of(self, kind, idx):
        """The rays a parameter can change: for a pose entry every ray near its box; for a
        payload voxel the rays passing within 1.05 cells of it (its trilinear support)."""
        k = idx[0]
        rays = self.S_k[k]
        if kind != "g_payload":
            return rays
        M = self.sc.M
        cell = 2.0 / (M - 1)
        centre = np.array([idx[3], idx[2], idx[1]], np.float64) * cell - 1.0  # (x, y, z) local
        ol = (self._ol[k] - centre) / cell
        dl = self._dl[k] / cell
        d = pair_depth(ol, dl, self.rays.t_near, self.rays.t_far)
        return rays[d <= 1.05]

    def near_kink(self, k, rays, i_last):
        """Rays (a subset of S_k) with a sample i <= i_last within KINK_BAND of a cell
        boundary (voxel units) or a face (local units) of primitive k, FP64."""
        r = self.rays
        pos = np.searchsorted(self.S_k[k], rays)
        ol, dl = self._ol[k][pos], self._dl[k][pos]
        n_steps = int(np.ceil((r.t_far - r.t_near) / r.dt - 1e-4))
        ts = float(r.t_near) + np.arange(n_steps) * float(r.dt)
        M = self.sc.M
        out = np.zeros(rays.size, bool)
        for a in range(0, rays.size, 2048):
            b = min(a + 2048, rays.size)
            y = ol[a:b, None, :] + ts[None, :, None] * dl[a:b, None, :]
            ym = np.abs(y).max(2)
            live = np.arange(n_steps)[None, :] <= i_last[a:b, None]
            u = (y + 1.0) * 0.5 * (M - 1)
            dcell = np.abs(u - np.round(u)).min(2)
            near = (np.abs(ym - 1.0) < KINK_BAND) | ((ym <= 1.0) & (dcell < KINK_BAND))
            out[a:b] = (near & live).any(1)
        return out

    def _perturbed(self, kind, idx, delta):
        sc = self.sc
        name = KEYS[kind]
        arr = getattr(sc, name).copy()
        v0 = arr[idx]
        arr[idx] = np.float32(np.float64(v0) + delta)
        actual = float(np.float64(arr[idx]) - np.float64(v0))
        kw = {"t": sc.t, "q": sc.q, "s": sc.s, "payload": sc.payload}
        kw[name] = arr
        return synthetic.Scene(M=sc.M, **kw), actual

    def per_ray(self, kind, idx, h0=H):
        """Per-ray central differences at h0 and h0/2 for the rays the parameter changes,
        which of them are smooth, and which of those are left out because their clamp
        sits within SAT_BAND of the neighbouring sample or (pose entries) a sample lies
        within KINK_BAND of a kink of the primitive's field. Returns (rays, fd_h0,
        smooth, at_sat); smooth excludes at_sat."""
        rays = self.rays_of(kind, idx)
        sub = self._sub(rays)
        tgt = self.target[rays]

        def lo(sc):
            r = oracle.render(sc, sub, F64M)
            return ((r["rgba"][:, :3] - tgt) ** 2).sum(1) / self.S.size, r["n_eval"]

        key = (kind, idx[0]) if kind != "g_payload" else (kind, idx)
        if key not in self._n0:
            r0 = oracle.render(self.sc, sub, F64M)
            beta = np.asarray(r0["beta"])
            at_sat = (np.asarray(r0["i_clamp"]) >= 0) & ((beta < SAT_BAND) | (beta > 1.0 - SAT_BAND))
            if kind != "g_payload":
                at_sat |= self.near_kink(idx[0], rays, np.asarray(r0["i_last"]))
            self._n0[key] = (r0["n_eval"], at_sat)
        n0, at_sat = self._n0[key]
        res = []
        for h in (h0, h0 / 2):
            sp, dp = self._perturbed(kind, idx, +h)
            sm, dm = self._perturbed(kind, idx, -h)
            lp, np_ = lo(sp)
            lm, nm = lo(sm)
            res.append(((lp - lm) / (dp - dm), (np_ == n0) & (nm == n0)))
        (f1, s1), (f2, s2) = res
        floor = 1e-3 * np.abs(f1).max(initial=0.0)
        agree = np.abs(f1 - f2) <= SMOOTH_TOL * np.maximum(np.abs(f1), floor)
        smooth = s1 & s2 & agree
        return rays, f1, smooth & ~at_sat, smooth & at_sat


def check(prob, whole_grads, grad_of_rays, params, label="", h=H):
    """whole_grads: the gradient tensors of the whole loss (for the C9 floor);
    grad_of_rays(kind, idx, rays) -> the gradient entry of the loss restricted to
    those rays. Returns (C9 errors, smooth-ray fractions, rows)."""
    scale = {k: float(np.abs(v).max()) for k, v in whole_grads.items()}
    rows, errs, fracs = [], [], []
    for kind, idx in params:
        rays, f1, smooth, at_sat = prob.per_ray(kind, idx, h)
        fd = float(f1[smooth].sum())
        cond = float(np.abs(f1[smooth]).sum())
        g = float(grad_of_rays(kind, idx, rays[smooth]))
        plain = abs(g - fd) / max(abs(fd), 1e-3 * scale[kind])
        err = abs(g - fd) / max(abs(fd), 1e-3 * scale[kind], FP32_FLOOR * cond)
        frac = float(smooth.mean()) if smooth.size else 1.0
        errs.append(err)
        fracs.append(frac)
        n_sat = int(at_sat.sum())
        rows.append((kind, idx, g, fd, err, int(smooth.size - smooth.sum()) - n_sat, int(smooth.size), n_sat,
                     plain, cond / max(abs(fd), 1e-300)))
    errs, fracs = np.asarray(errs), np.asarray(fracs)
    plains = np.asarray([r[8] for r in rows])
    from parity_rules import REPORT

    REPORT.append(("fd", label, {"params": len(params), "err_max": float(errs.max()),
                                 "plain_c9_max": float(plains.max()), "plain_c9_ok": int((plains <= TOL).sum()),
                                 "kinked": sum(r[5] for r in rows), "near_kink": sum(r[7] for r in rows),
                                 "rays": sum(r[6] for r in rows)}))
    print(f"FD check {label}: {len(params)} parameters, error max {errs.max():.3e} median "
          f"{np.median(errs):.3e}; plain C9 (no conditioning floor) max {plains.max():.3e}, "
          f"{int((plains <= TOL).sum())} of {len(params)} within {TOL}; rays straddling a kink: "
          f"{sum(r[5] for r in rows)} of {sum(r[6] for r in rows)}, within FP32 rounding of a kink: "
          f"{sum(r[7] for r in rows)} (parameter with the most left out: {1 - fracs.min():.3f})")
    for r in rows:
        if r[8] > TOL:
            print("   ", r[0], r[1], f"g={r[2]:.6e} fd={r[3]:.6e} err={r[4]:.2e} plain C9 {r[8]:.2e} "
                  f"sum|fd_r|/|fd| {r[9]:.1f} kinked rays {r[5]}/{r[6]}, near a kink {r[7]}")
    return errs, fracs, rows
