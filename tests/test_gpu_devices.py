"""Two devices in one process: the kernels' dynamic shared-memory opt-in belongs to
one context, so the library remembers it per (kernel, context). A render on device 1
after one on device 0 (the 128+ KB one-block BVH sort, the frame kernel and the
adjoint) must opt in again there and give the same image and gradients. Skipped
where the process sees fewer than two GPUs."""
import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2103_01954_gb300 import torch_ops as T  # noqa: E402


def _render(dev_index, sc, rays, g):
    dev = torch.device("cuda", dev_index)
    with torch.cuda.device(dev):
        ctx = T.Context(dev_index)
        up = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        t, q, s, p = up(sc.t), up(sc.q), up(sc.s), up(sc.payload)
        prims = T.prims_struct(t, q, s, p)
        rs = T.rays_struct(up(rays.o), up(rays.d), t_near=rays.t_near, t_far=rays.t_far, dt=rays.dt,
                           eps_early=0.0, bg=(0.0, 0.0, 0.0), width=rays.width, height=rays.height)
        bvh = T.BVH(ctx)
        bvh.build(prims)
        out, saved = T.raymarch_fwd(ctx, prims, bvh, rs, want_saved=True)
        gp = torch.zeros(p.shape, dtype=torch.float32, device=dev)
        gt, gq, gs = torch.zeros_like(t), torch.zeros_like(q), torch.zeros_like(s)
        T.raymarch_bwd(ctx, prims, bvh, rs, saved, up(g), gp, gt, gq, gs)
        ctx.sync()
        return out.cpu().numpy(), gp.cpu().numpy(), gt.cpu().numpy()


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs two GPUs in one process")
def test_render_on_two_devices_in_one_process():
    sc, rays, _ = synthetic.make_config("small_4096x16^3_83x128", 0)
    g = np.random.default_rng(1).standard_normal((rays.n, 4)).astype(np.float32)
    a = _render(0, sc, rays, g)
    b = _render(1, sc, rays, g)
    np.testing.assert_array_equal(a[0], b[0])
    for x, y in zip(a[1:], b[1:]):
        assert np.abs(x - y).max() <= 1e-5 * max(np.abs(x).max(), 1e-30)
