"""Benchmark of the MVP ray-march path on GB300.

One step = one frame of the paper-scale workload (4096 primitives of 16^3 RGBA FP32
voxels on an ellipsoid shell, one 667x1024 camera, dt = 0.005 over t in [1, 5]):
rebuild the BVH (per-frame rebuild, Sec. 3.2.1) and march every pixel (Sec. 3.2.2),
through the C ABI. Inputs are resident in HBM; L2 is flushed (a 512 MiB write)
before every timed step and each step is timed with CUDA events on its stream.

Printed: one JSON line (rank 0). Besides the headline forward FP32 figure it carries
the BF16 / FP16 payload variants, the 512x32^3 and 32768x8^3 sweeps, and the
differentiation workload (512 x 32^3, 4 cameras of 512x512, forward + backward).

--impl reference times the CPU oracle (FP64, plain loops; the only reference this
method has) on a bounded ray sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "paper_4096x16^3_667x1024"
METRIC = "MVP raymarch Mrays/s fwd & fwd+bwd vs plain FP32; serving p50/p99 ms/frame"
# resident 4-warp blocks per SM of the march and adjoint kernels (their launch bounds;
# registers allow no more): the residency the gather probe is also run at
MARCH_BLOCKS_PER_SM = 5
ADJOINT_BLOCKS_PER_SM = 3

# Algorithmic work per (sample, primitive) evaluation: 8 voxel reads of 4 channels
# (bytes by dtype) and the FP32 operations of the definition (local coordinates
# 3x3 FMA = 18, trilinear 7 lerps x 4 channels x 3 = 84, accumulation 7).
FLOP_PER_EVAL = 109
GATHER_BYTES = {"f32": 128, "bf16": 64, "f16": 64}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def aggregate(ms_local: float, rays_local: int, world: int, device=None) -> tuple[float, float]:
    """Weak scaling over ranks: every rank renders its own frame; the job's step time
    is the slowest rank's, and the value counts the rays of all ranks.
    Returns (ms_per_step, Mrays/s). Collective only when world > 1."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist

        tt = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    return ms, world * rays_local / (ms * 1e-3) / 1e6


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region.

    Each sample carries nvidia-smi's own timestamp; the summary keeps those taken between
    the region's start and end (host wall clock), so it does not depend on when the
    samples reach the file. The region starts once nvidia-smi has written its first
    sample (bounded wait), so its start-up does not eat the region. A region shorter
    than the sampling interval holds no sample; then the last sample before it and the
    first after it stand in, labelled as such."""

    QUERY = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int, interval_ms: int = 50, start_timeout_s: float = 5.0):
        self.index = index
        self.interval_ms = interval_ms
        self.start_timeout_s = start_timeout_s
        self.proc = None
        self.t0 = self.t1 = 0.0  # the region, host wall clock (s)
        # the raw samples go to $MVP_BENCH_OUT (default: the system's temporary directory)
        out_dir = os.environ.get("MVP_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)],
                stdout=self.f, stderr=subprocess.DEVNULL)
            t_end = time.monotonic() + self.start_timeout_s
            while os.path.getsize(self.path) == 0 and time.monotonic() < t_end and self.proc.poll() is None:
                time.sleep(0.005)
        except Exception:
            self.proc = None
        self.t0 = time.time()
        return self

    def __exit__(self, *a):
        self.t1 = time.time()
        if self.proc is not None:
            time.sleep(3 * self.interval_ms / 1e3)  # a sample after the region
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    @staticmethod
    def _when(stamp: str):
        import datetime

        try:
            return datetime.datetime.strptime(stamp.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            r = [x.strip() for x in line.split(",")]
            if len(r) >= 8 and self._when(r[0]) is not None:
                rows.append((self._when(r[0]), r[1:]))
        window = "timed region"
        sel = [r for ts, r in rows if self.t0 <= ts <= self.t1]
        if not sel:
            before = [r for ts, r in rows if ts < self.t0][-1:]
            after = [r for ts, r in rows if ts > self.t1][:1]
            sel = before + after
            window = "bracketing the timed region (shorter than the sampling interval)"
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in sel if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in sel if r[1].replace(".", "").isdigit()]
        reasons = sorted({self.REASONS[i] for r in sel for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sel), "window": window, "interval_ms": self.interval_ms}


def _frame_runner(cfg: str, seed: int, dtype: str, want_bwd: bool, torch, T, synthetic, sequential=False,
                  schedule=True):
    """Set up a workload on the device; returns (step(), n_rays, info). sequential:
    blend each ray's saturating sample in BVH order (MVP_BLEND_SEQUENTIAL); schedule:
    the library's cost-ordered tile schedule (off: the plain tile order)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    scene, rays, extra = synthetic.make_config(cfg, seed)
    ctx = T.Context(dev.index)
    ctx.set_tile_schedule(schedule)
    t = torch.from_numpy(scene.t).to(dev)
    q = torch.from_numpy(scene.q).to(dev)
    s = torch.from_numpy(scene.s).to(dev)
    p32 = torch.from_numpy(scene.payload).to(dev)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    payload = p32 if dtype == "f32" else T.pack_payload(ctx, p32, tdt)
    if dtype != "f32":
        del p32
    o = torch.from_numpy(rays.o).to(dev)
    d = torch.from_numpy(rays.d).to(dev)
    prims = T.prims_struct(t, q, s, payload)
    rs = T.rays_struct(o, d, t_near=rays.t_near, t_far=rays.t_far, dt=rays.dt, eps_early=rays.eps_early,
                       bg=tuple(rays.bg), width=rays.width, height=rays.height, sequential=sequential)
    bvh = T.BVH(ctx)
    bvh.build(prims)
    out = torch.empty((rays.n, 4), dtype=torch.float32, device=dev)
    saved = torch.empty(T.saved_bytes(rays.n), dtype=torch.uint8, device=dev) if want_bwd else None
    grads = None
    if want_bwd:
        target = torch.from_numpy(extra["target"]).to(dev)
        gp = torch.zeros(payload.shape, dtype=torch.float32, device=dev)
        gt, gq, gs = torch.zeros_like(t), torch.zeros_like(q), torch.zeros_like(s)
        grad_out = torch.zeros((rays.n, 4), dtype=torch.float32, device=dev)
        grads = (gp, gt, gq, gs, grad_out, target)
    ev = {"march": [], "bwd": []}
    # the ABI structs hold raw device pointers: the step keeps their tensors alive
    keep = (t, q, s, payload, o, d)

    def step(time_march=False):
        assert keep
        bvh.build(prims)
        if time_march:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
        T.raymarch_fwd(ctx, prims, bvh, rs, out=out, saved=saved)
        if time_march:
            e1.record()
            ev["march"].append((e0, e1))
        if want_bwd:
            gp, gt, gq, gs, grad_out, target = grads
            # photometric L2 loss (Sec. 3.3, lambda = 1): dL/dI = 2 (I - target) / R
            torch.sub(out[:, :3], target, out=grad_out[:, :3]).mul_(2.0 / rays.n)
            gp.zero_(), gt.zero_(), gq.zero_(), gs.zero_()
            if time_march:
                b0 = torch.cuda.Event(enable_timing=True)
                b1 = torch.cuda.Event(enable_timing=True)
                b0.record()
            T.raymarch_bwd(ctx, prims, bvh, rs, saved, grad_out, gp, gt, gq, gs)
            if time_march:
                b1.record()
                ev["bwd"].append((b0, b1))

    info = {"scene": scene, "rays": rays, "ctx": ctx, "prims": prims, "bvh": bvh, "rs": rs, "ev": ev, "o": o, "d": d, "keep": keep,
            "payload_bytes": payload.numel() * payload.element_size(), "out": out,
            "host": (scene, rays), "n_prims": int(scene.t.shape[0]), "M": int(scene.M)}
    return step, rays.n, info


def _time_steps(torch, step, steps, warmup, flush, time_march=False):
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    durs = []
    for _ in range(steps):
        flush.fill_(1.0)  # write 512 MiB: evicts L2 between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step(time_march) if time_march else step()
        e1.record()
        durs.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in durs]


def _e2e(torch, T, info, steps, warmup, payload_dtype="f32", rays_from="camera"):
    """The same frame through the C ABI from pinned host buffers: every step copies its
    inputs (poses, payload) host->device, makes the camera's rays on the device
    (rays_from="camera": the frame's input is the 3x4 camera and focal length, passed
    by value) or copies precomputed rays from the host (rays_from="host"), builds the
    BVH, marches, and reads the image back to pinned host memory. Frames are pipelined
    as a streaming renderer would run them: frame k+1's inputs are copied on a copy
    stream (into the other of two device buffer sets) while frame k renders, and each
    image is read back on a third stream. The serial time (one stream, nothing
    overlapped) is reported beside."""
    scene, rays = info["host"]
    dev = torch.device("cuda", torch.cuda.current_device())
    cam = rays.cameras[0] if rays_from == "camera" else None
    c2w = cam.matrix34() if cam else None
    arrays = (scene.t, scene.q, scene.s, scene.payload) + (() if cam else (rays.o, rays.d))
    hs = [torch.from_numpy(a).pin_memory() for a in arrays]
    if payload_dtype != "f32":
        # the host holds the payload in the reduced type (packed once by mvp_pack_payload)
        tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[payload_dtype]
        hs[3] = T.pack_payload(info["ctx"], hs[3].to(dev), tdt).cpu().pin_memory()
    sets = []
    for _ in range(2):
        ds = [torch.empty(h.shape, dtype=h.dtype, device=dev) for h in hs]
        if cam:  # the rays' device buffers, filled from the camera every frame
            ds += [torch.empty((rays.n, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        prims = T.prims_struct(ds[0], ds[1], ds[2], ds[3])
        rs = T.rays_struct(ds[4], ds[5], t_near=rays.t_near, t_far=rays.t_far, dt=rays.dt, width=rays.width,
                           height=rays.height)
        out = torch.empty((rays.n, 4), dtype=torch.float32, device=dev)
        hout = torch.empty((rays.n, 4), dtype=torch.float32).pin_memory()
        sets.append({"ds": ds, "prims": prims, "rs": rs, "out": out, "hout": hout,
                     "copied": torch.cuda.Event(), "rendered": torch.cuda.Event(), "read": torch.cuda.Event()})
    ctx, bvh = info["ctx"], info["bvh"]
    comp = torch.cuda.current_stream()
    copy_s, read_s = torch.cuda.Stream(), torch.cuda.Stream()
    for st in sets:  # both sets start free
        st["rendered"].record(comp)
        st["read"].record(comp)

    def step(k):
        st = sets[k % 2]
        with torch.cuda.stream(copy_s):
            copy_s.wait_event(st["rendered"])  # the set's previous frame no longer reads its inputs
            for h, d in zip(hs, st["ds"]):
                d.copy_(h, non_blocking=True)
            st["copied"].record(copy_s)
        comp.wait_event(st["copied"])
        comp.wait_event(st["read"])  # the set's previous image has been read back
        if cam:
            T.camera_rays(ctx, c2w, cam.focal, rays.width, rays.height, out=(st["ds"][4], st["ds"][5]))
        bvh.build(st["prims"])
        T.raymarch_fwd(ctx, st["prims"], bvh, st["rs"], out=st["out"])
        st["rendered"].record(comp)
        with torch.cuda.stream(read_s):
            read_s.wait_event(st["rendered"])
            st["hout"].copy_(st["out"], non_blocking=True)
            st["read"].record(read_s)

    def serial_step():
        st = sets[0]
        for h, d in zip(hs, st["ds"]):
            d.copy_(h, non_blocking=True)
        if cam:
            T.camera_rays(ctx, c2w, cam.focal, rays.width, rays.height, out=(st["ds"][4], st["ds"][5]))
        bvh.build(st["prims"])
        T.raymarch_fwd(ctx, st["prims"], bvh, st["rs"], out=st["out"])
        st["hout"].copy_(st["out"], non_blocking=True)

    def timed(fn, n):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(comp)
        for k in range(n):
            fn(k)
        comp.wait_stream(copy_s)
        comp.wait_stream(read_s)
        e1.record(comp)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    for k in range(warmup):
        step(k)
    ms = timed(step, steps)
    for _ in range(warmup):
        serial_step()
    ms_serial = timed(lambda k: serial_step(), steps)
    ctx.sync()
    # the streamed frames must equal the frame rendered from the resident inputs (of
    # the same payload type; with the camera's rays when the frame makes its own)
    bvh.build(info["prims"])
    rs_ref = info["rs"]
    if cam:
        o, d = T.camera_rays(ctx, c2w, cam.focal, rays.width, rays.height)
        rs_ref = T.rays_struct(o, d, t_near=rays.t_near, t_far=rays.t_far, dt=rays.dt, width=rays.width,
                               height=rays.height)
    T.raymarch_fwd(ctx, info["prims"], bvh, rs_ref, out=info["out"])
    ctx.sync()
    ref = info["out"].cpu()
    same = all(torch.equal(st["hout"], ref) for st in sets)
    h2d = sum(h.numel() * h.element_size() for h in hs) + (13 * 4 if cam else 0)  # + camera and focal
    d2h = rays.n * 4 * 4
    return {"value": rays.n / (ms * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": ms, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "serial_ms_per_step": ms_serial,
            "serial_value": rays.n / (ms_serial * 1e-3) / 1e6,
            "pipeline": "frame k+1's inputs copied (copy stream, second buffer set) while frame k renders; "
                        "images read back on a third stream; every copy inside the timed region",
            "payload_dtype": payload_dtype, "image_matches_resident_frame": bool(same),
            "rays": "made on the device from the frame's camera (48 + 4 bytes in)" if cam
            else "copied from the host every frame"}


def _host_threads() -> int:
    """Host cores this process may run on; the oracle is given exactly this many threads."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _cpu_baseline(seconds: float = 15.0):
    """The oracle (FP64, pruned mode, FP32 membership) on a seeded ray sample of the
    workload, on all host cores."""
    import oracle
    import synthetic

    oracle.build()
    scene, rays, _ = synthetic.make_config(WORKLOAD, 0)
    rng = np.random.default_rng(123)
    n = 256
    cores = _host_threads()
    total_rays, total_s = 0, 0.0
    while total_s < seconds:
        sel = rng.choice(rays.n, n, replace=False)
        sub = synthetic.Rays(o=rays.o[sel], d=rays.d[sel], t_near=rays.t_near, t_far=rays.t_far, dt=rays.dt)
        t0 = time.perf_counter()
        oracle.render(scene, sub, n_threads=cores)
        dt = time.perf_counter() - t0
        total_rays += n
        total_s += dt
        if dt < seconds / 8:
            n *= 2
    # the whole tiny frame (8 primitives of 8^3, 64x64), as a second reference point
    s0, r0, _ = synthetic.make_config("tiny_8x8^3_64x64", 0)
    t0 = time.perf_counter()
    oracle.render(s0, r0, n_threads=cores)
    tiny_s = time.perf_counter() - t0
    return {"value": total_rays / total_s / 1e6, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
            "tiny_8x8^3_64x64_full_frame": {"seconds": round(tiny_s, 4),
                                            "mrays_per_s": round(r0.n / tiny_s / 1e6, 4)},
            "sample": f"{total_rays} rays in batches of seeded random pixels of the 667x1024 frame (683008 "
                      f"pixels; batches drawn independently, so pixels may repeat), FP64 oracle, pruned mode, "
                      f"{cores} OpenMP threads, {total_s:.1f} s"}


def _ncu_record(kernel_key: str) -> dict:
    """The committed ncu figures of a kernel (profiles/traffic.json), if they were taken
    with the kernel's current sources (the digest of the files the record lists), else {}."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return {}
    try:
        from paper_2103_01954_gb300 import build as b

        e = json.load(open(p)).get(kernel_key)
        if e and e.get("source_digest") == b.sources_digest(e["sources"]):
            return e
    except Exception:
        return {}
    return {}


def _orbit(torch, T, synthetic, args, flush, n_views=8, deg=0.5):
    """The paper frame seen by a camera that orbits the avatar by `deg` degrees per
    frame (rays made on the device per view beforehand), so every frame's tile
    schedule comes from the previous, different view: the rate with the schedule and
    with the plain tile order."""
    out = {"views": n_views, "deg_per_frame": deg, "workload": WORKLOAD}
    for sched in (True, False):
        st, nr, inf = _frame_runner(WORKLOAD, 0, "f32", False, torch, T, synthetic, schedule=sched)
        r = inf["rays"]
        cam = r.cameras[0]
        W, H = r.width, r.height
        eye0 = np.asarray(cam.eye, np.float64)
        rs = []
        keep = []
        for v in range(n_views):
            a = np.deg2rad(deg * v)
            rot = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
            c = synthetic.look_at_camera(rot @ eye0, W, H, cam.focal)
            o, d = T.camera_rays(inf["ctx"], c.matrix34(), cam.focal, W, H)
            keep.append((o, d))
            rs.append(T.rays_struct(o, d, t_near=r.t_near, t_far=r.t_far, dt=r.dt, width=W, height=H))
        frame = [0]

        def step():
            inf["bvh"].build(inf["prims"])
            T.raymarch_fwd(inf["ctx"], inf["prims"], inf["bvh"], rs[frame[0] % n_views], out=inf["out"])
            frame[0] += 1

        d = _time_steps(torch, step, args.steps, args.warmup, flush)
        inf["ctx"].sync()
        m = float(np.mean(d))
        out["value_scheduled" if sched else "value_plain_order"] = round(nr / (m * 1e-3) / 1e6, 3)
        out["ms_scheduled" if sched else "ms_plain_order"] = round(m, 4)
        del st, inf, keep, rs
        torch.cuda.empty_cache()
    out["unit"] = "Mrays/s"
    return out


def _sequential_blend(torch, T, synthetic, args, flush):
    """The headline frame with the paper-literal blend (the primitives at a ray's
    saturating sample taken one by one in BVH order): its rate, and how far its image
    is from the summed rule's on the same frame."""
    st, nr, inf = _frame_runner(WORKLOAD, 0, "f32", False, torch, T, synthetic, sequential=True)
    d = _time_steps(torch, st, args.steps, args.warmup, flush, time_march=True)
    inf["ctx"].sync()
    m = float(np.mean(d))
    mm = float(np.mean([a.elapsed_time(b) for a, b in inf["ev"]["march"]]))
    seq = inf["out"].clone()
    r = inf["rays"]
    rs = T.rays_struct(inf["o"], inf["d"], t_near=r.t_near, t_far=r.t_far, dt=r.dt, eps_early=r.eps_early,
                       bg=tuple(r.bg), width=r.width, height=r.height)
    summ = torch.empty_like(seq)
    T.raymarch_fwd(inf["ctx"], inf["prims"], inf["bvh"], rs, out=summ)
    inf["ctx"].sync()
    diff = (seq - summ).abs().amax(dim=1)
    out = {"value": round(nr / (m * 1e-3) / 1e6, 3), "unit": "Mrays/s", "ms_per_step": round(m, 4),
           "march_ms": round(mm, 4), "workload": WORKLOAD, "payload_dtype": "f32",
           "pixels_differing_from_summed_1e-3": round(float((diff > 1e-3).float().mean()), 4),
           "max_abs_diff_from_summed": round(float(diff.max()), 5),
           "alpha_max_abs_diff": float((seq[:, 3] - summ[:, 3]).abs().max())}
    del st, inf, seq, summ
    torch.cuda.empty_cache()
    return out


def _vr_stereo(torch, T, synthetic, flush, steps=20, view_dependent=False):
    """The paper's live binocular viewer workload (Sec. 4: two 896x832 views at 40 Hz):
    per frame the primitives move (two pose sets alternate), the BVH is rebuilt once and
    both eyes (6.4 cm apart) are rendered in one launch over the stacked [2][832][896]
    image. Headless: the images stay on the device. view_dependent: each frame also
    assembles its payload (BF16, faded) from that frame's view-dependent colour (two
    decoded colour sets alternate, standing in for the colour decoder's per-frame
    output) and the shared opacity, as the paper's viewer decodes one payload per frame."""
    dev = torch.device("cuda", torch.cuda.current_device())
    W, H = 896, 832
    sc, _, _ = synthetic.make_config(WORKLOAD, 0)
    ctx = T.Context(dev.index)
    rng = np.random.default_rng(40)
    ts = [torch.from_numpy(sc.t).to(dev),
          torch.from_numpy(sc.t + rng.normal(0, 0.005, sc.t.shape).astype(np.float32)).to(dev)]
    q = torch.from_numpy(sc.q).to(dev)
    s = torch.from_numpy(sc.s).to(dev)
    p = torch.from_numpy(sc.payload).to(dev)
    cam = synthetic.random_camera(rng, 3.0, W, H, 900.0)
    if view_dependent:
        # object-centric view vectors of two consecutive frames (the head moved 2 cm)
        eye = cam.eye.astype(np.float64)
        views = [-eye, -(eye + 0.02 * cam.c2w[:, 0])]
        rgbs = [torch.from_numpy(synthetic.view_colors(sc, v, seed=0)).to(dev) for v in views]
        op = torch.from_numpy(np.ascontiguousarray(sc.payload[..., 3])).to(dev)
        p = torch.empty(sc.payload.shape, dtype=torch.bfloat16, device=dev)
    left = cam.matrix34()
    right = left.copy()
    right[:, 3] += 0.064 * right[:, 0]
    o = torch.empty((2 * H * W, 3), dtype=torch.float32, device=dev)
    d = torch.empty_like(o)
    for eye, c in enumerate((left, right)):
        oe, de = T.camera_rays(ctx, c, 900.0, W, H)
        o[eye * H * W:(eye + 1) * H * W] = oe
        d[eye * H * W:(eye + 1) * H * W] = de
    rs = T.rays_struct(o, d, t_near=1.0, t_far=5.0, dt=0.005, width=W, height=2 * H)
    out = torch.empty((2 * H * W, 4), dtype=torch.float32, device=dev)
    bvh = T.BVH(ctx)
    prims = [T.prims_struct(t, q, s, p) for t in ts]

    frame = [0]

    decode = [view_dependent]

    def step():
        pr = prims[frame[0] % 2]  # the primitives moved since the last frame
        if decode[0]:  # this frame's payload, into the buffer the prims point at
            T.assemble_payload(ctx, rgbs[frame[0] % 2], op, torch.bfloat16, 8.0, 8, out=p)
        frame[0] += 1
        bvh.build(pr)
        T.raymarch_fwd(ctx, pr, bvh, rs, out=out)

    durs = _time_steps(torch, step, steps, 3, flush)
    ctx.sync()
    ms = float(np.mean(durs))
    res = {"ms_per_frame_pair": round(ms, 4), "hz": round(1000.0 / ms, 1), "target_hz": 40,
           "mrays_per_s": round(2 * H * W / (ms * 1e-3) / 1e6, 2), "views": "2 x 896x832, 6.4 cm apart",
           "step": "BVH rebuild (moved primitives) + both eyes in one launch", "workload": WORKLOAD}
    if view_dependent:
        # the same loop on the last assembled payload, kept: the difference is the
        # per-frame assembly (the faded opacity itself lengthens the march)
        decode[0] = False
        ms_static = float(np.mean(_time_steps(torch, step, steps, 3, flush)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        am = []
        for i in range(10):
            flush.fill_(1.0)
            e0.record()
            T.assemble_payload(ctx, rgbs[i % 2], op, torch.bfloat16, 8.0, 8, out=p)
            e1.record()
            e1.synchronize()
            am.append(e0.elapsed_time(e1))
        a_ms = float(np.mean(am))
        nv = p.numel() // 4
        res.update({"step": "assemble the frame's BF16 payload (view colour + faded shared opacity) + BVH rebuild "
                            "(moved primitives) + both eyes in one launch",
                    "payload_dtype": "bf16", "assemble_ms": round(a_ms, 4),
                    "ms_per_frame_pair_payload_kept": round(ms_static, 4),
                    "assemble_GBps": round(nv * 24 / (a_ms * 1e-3) / 1e9, 1)})
    return res


def _fade_pack(torch, T, synthetic, peaks):
    """The opacity fade fused with the FP32 -> BF16 payload conversion on the
    paper-scale payload (4096 x 16^3 voxels): 16 bytes read and 8 written per voxel,
    against the measured HBM copy bandwidth."""
    dev = torch.device("cuda", torch.cuda.current_device())
    sc, _, _ = synthetic.make_config(WORKLOAD, 0)
    ctx = T.Context(dev.index)
    p32 = torch.from_numpy(sc.payload).to(dev)
    out = torch.empty(p32.shape, dtype=torch.bfloat16, device=dev)
    for _ in range(3):
        T.fade_payload(ctx, p32, torch.bfloat16, 8.0, 8, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 20
    e0.record()
    for _ in range(n):
        T.fade_payload(ctx, p32, torch.bfloat16, 8.0, 8, out=out)
    e1.record()
    torch.cuda.synchronize()
    ctx.sync()
    ms = e0.elapsed_time(e1) / n
    n_vox = p32.numel() // 4
    gbps = 24.0 * n_vox / (ms * 1e-3) / 1e9
    return {"ms": round(ms, 4), "GBps": round(gbps, 1),
            "hbm_frac": round(gbps / peaks["hbm_gbs"], 3) if peaks.get("hbm_gbs") else None,
            "bytes_per_voxel": 24, "voxels": n_vox, "workload": WORKLOAD}


def _pack(torch, T, synthetic, peaks):
    """The FP32 -> BF16 / FP16 payload conversion (mvp_pack_payload) on the paper-scale
    payload (4096 x 16^3 voxels): 16 bytes read and 8 written per voxel, against the
    measured HBM copy bandwidth."""
    dev = torch.device("cuda", torch.cuda.current_device())
    sc, _, _ = synthetic.make_config(WORKLOAD, 0)
    ctx = T.Context(dev.index)
    p32 = torch.from_numpy(sc.payload).to(dev)
    n_vox = p32.numel() // 4
    res = {"bytes_per_voxel": 24, "voxels": n_vox, "workload": WORKLOAD}
    for name, tdt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        for _ in range(3):
            out = T.pack_payload(ctx, p32, tdt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 20
        e0.record()
        for _ in range(n):
            out = T.pack_payload(ctx, p32, tdt)
        e1.record()
        torch.cuda.synchronize()
        ctx.sync()
        ms = e0.elapsed_time(e1) / n
        gbps = 24.0 * n_vox / (ms * 1e-3) / 1e9
        res[name] = {"ms": round(ms, 4), "GBps": round(gbps, 1),
                     "hbm_frac": round(gbps / peaks["hbm_gbs"], 3) if peaks.get("hbm_gbs") else None}
        del out
    return res


def _serve_trace(T, srv, ids, reqs, arrivals):
    """Submit `reqs` at their Poisson arrival times and poll until all are done.
    Returns (latencies in ms, wall seconds)."""
    import time as _t

    lat, pend = [], {}
    t0 = _t.perf_counter()
    j, n_req = 0, len(reqs)
    while j < n_req or pend:
        now = _t.perf_counter() - t0
        while j < n_req and arrivals[j] <= now:
            a, cam, w, h = reqs[j]
            pend[srv.submit_raw(T.Server.request(ids[a], cam.matrix34(), cam.focal, w, h, 1.0, 5.0, 0.005))] = j
            j += 1
        for tk in list(pend):
            st, ms = srv.poll(tk)
            if st == 0:
                lat.append(ms)
                del pend[tk]
    return lat, _t.perf_counter() - t0


def _serving_budget_run(torch, T, synthetic, ctx, av_bf16, av_f32, seed):
    """A 64 MB budget for images in flight on top of the 8 resident BF16 avatars: a
    64-request burst is admitted as memory frees up (the rest waits, none is lost), an
    extra FP32 avatar and a 4096x4096 request are refused (MVP_ERR_CAPACITY)."""
    from paper_2103_01954_gb300 import binding as B

    probe = T.Server(ctx, hbm_budget=100 * 10**9, max_slots=4)
    for a in av_bf16:
        probe.register(*a)
    resident = probe.stats()["resident_bytes"]
    probe.close()
    budget = resident + (64 << 20)
    srv = T.Server(ctx, hbm_budget=budget, max_slots=64)
    ids = [srv.register(*a) for a in av_bf16]
    refused_avatar = False
    try:
        srv.register(*av_f32[0])
    except B.MVPError as e:
        if e.status != B.MVP_ERR_CAPACITY:
            raise
        refused_avatar = True
    rng = np.random.default_rng(seed + 64)
    tks = []
    for j in range(64):
        w, h = synthetic.SERVE_RESOLUTIONS[j % 3]
        cam = synthetic.random_camera(rng, 3.0, w, h, float(max(w, h)))
        tks.append(srv.submit_raw(T.Server.request(ids[j % len(ids)], cam.matrix34(), cam.focal, w, h,
                                                   1.0, 5.0, 0.005)))
    pending_after_burst = srv.stats()["pending"]
    refused_request = False
    try:
        srv.submit_raw(T.Server.request(ids[0], cam.matrix34(), 4096.0, 4096, 4096, 1.0, 5.0, 0.005))
    except B.MVPError as e:
        if e.status != B.MVP_ERR_CAPACITY:
            raise
        refused_request = True
    done = 0
    for tk in tks:
        st, _ = srv.wait(tk, 60000.0)
        done += int(st == 0)
    st_ = srv.stats()
    srv.close()
    return {"hbm_budget": int(budget), "resident_bytes": int(resident), "image_budget": 64 << 20,
            "extra_f32_avatar_refused": refused_avatar, "burst_requests": 64,
            "pending_after_burst": int(pending_after_burst), "completed": done,
            "max_in_flight": int(st_["max_in_flight"]), "request_4096x4096_refused": refused_request,
            "device_status": int(st_["device_status"])}


def _serving(torch, T, synthetic, rates, n_req, seed=0):
    """Poisson arrivals over 8 resident BF16 avatars (512x32^3 ... 32768x8^3), random
    cameras on the radius-3 sphere, resolutions {256x256, 512x512, 667x1024}; served
    with continuous batching (mvp_serve_*) and, on the same trace, one request at a
    time with FP32 payloads (mvp_camera_rays + mvp_raymarch_fwd, synchronised). At the
    highest rate the same trace is also served with FP32 payloads; a 64 MB budget run
    exercises refusal."""
    import time as _t

    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = T.Context(dev.index)
    av_bf16, av_f32, bvhs = [], [], []
    for i in range(len(synthetic.AVATARS)):
        sc = synthetic.make_avatar(i, seed)
        t = torch.from_numpy(sc.t).to(dev)
        q = torch.from_numpy(sc.q).to(dev)
        s = torch.from_numpy(sc.s).to(dev)
        p32 = torch.from_numpy(sc.payload).to(dev)
        av_f32.append((t, q, s, p32))
        av_bf16.append((t, q, s, T.pack_payload(ctx, p32, torch.bfloat16)))
        bvh = T.BVH(ctx)
        bvh.build(T.prims_struct(t, q, s, p32))
        bvhs.append(bvh)
    srv = T.Server(ctx, hbm_budget=100 * 10**9, max_slots=64, arena_bytes=2 << 30)
    ids = [srv.register(*a) for a in av_bf16]
    resident = srv.stats()["resident_bytes"]
    ids32 = [srv.register(*a) for a in av_f32]
    out_buf = torch.empty((1024 * 667, 4), dtype=torch.float32, device=dev)
    results = {}
    for ri, rate in enumerate(rates):
        rng = np.random.default_rng(seed + int(rate))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
        reqs = []
        for j in range(n_req):
            a = int(rng.integers(0, len(ids)))
            w, h = synthetic.SERVE_RESOLUTIONS[int(rng.integers(0, 3))]
            cam = synthetic.random_camera(rng, 3.0, w, h, float(max(w, h)))
            reqs.append((a, cam, w, h))
        rays = sum(w * h for _, _, w, h in reqs)
        # warm-up: a few requests so kernels and arenas are resident
        for a, cam, w, h in reqs[:4]:
            for table in (ids, ids32):
                tk = srv.submit_raw(T.Server.request(table[a], cam.matrix34(), cam.focal, w, h, 1.0, 5.0, 0.005))
                srv.wait(tk, 60000.0)
        # continuous batching, BF16 payloads
        lat, wall = _serve_trace(T, srv, ids, reqs, arrivals)
        st_ = srv.stats()
        # one request at a time, FP32 payloads, same trace
        lat1 = []
        t0 = _t.perf_counter()
        for k, (a, cam, w, h) in enumerate(reqs):
            while _t.perf_counter() - t0 < arrivals[k]:
                pass
            tt, qq, ss, pp = av_f32[a]
            prims = T.prims_struct(tt, qq, ss, pp)
            o, d = T.camera_rays(ctx, cam.matrix34(), cam.focal, w, h)
            rs = T.rays_struct(o, d, t_near=1.0, t_far=5.0, dt=0.005, width=w, height=h)
            T.raymarch_fwd(ctx, prims, bvhs[a], rs, out=out_buf[: w * h])
            torch.cuda.current_stream().synchronize()
            lat1.append((_t.perf_counter() - t0 - arrivals[k]) * 1e3)
        wall1 = _t.perf_counter() - t0
        ctx.sync()
        r = {"requests": n_req, "p50_ms": round(float(np.percentile(lat, 50)), 3),
             "p99_ms": round(float(np.percentile(lat, 99)), 3), "mrays_per_s": round(rays / wall / 1e6, 2),
             "max_in_flight": int(st_["max_in_flight"]), "device_status": int(st_["device_status"]),
             "one_at_a_time_f32": {"p50_ms": round(float(np.percentile(lat1, 50)), 3),
                                   "p99_ms": round(float(np.percentile(lat1, 99)), 3),
                                   "mrays_per_s": round(rays / wall1 / 1e6, 2)}}
        if ri == len(rates) - 1:
            # the same trace through the same server with FP32 payloads
            lat32, wall32 = _serve_trace(T, srv, ids32, reqs, arrivals)
            r["served_f32_payload"] = {"p50_ms": round(float(np.percentile(lat32, 50)), 3),
                                       "p99_ms": round(float(np.percentile(lat32, 99)), 3),
                                       "mrays_per_s": round(rays / wall32 / 1e6, 2)}
        results[f"{rate}_req_per_s"] = r
    srv.close()
    budget_run = _serving_budget_run(torch, T, synthetic, ctx, av_bf16, av_f32, seed)
    return {"avatars": [f"{n}x{M}^3" for n, M, _ in synthetic.AVATARS], "payload": "bf16",
            "resident_bytes": int(resident), "hbm_budget": 100 * 10**9,
            "resolutions": ["256x256", "512x512", "667x1024"], "latency": "host time from submit to completion seen",
            "rates": results, "budget_64MB_images": budget_run}


def _gather_probe(torch, T):
    """Ceilings of the march's voxel access pattern on this GPU (mvp_gather_probe):
    8-corner gathers (FP32 16-byte and BF16 8-byte voxels; plain layout, and the
    duplicated x-pair and xy-quad layouts that fetch a cell in 4 or 2 loads, and the
    plain layout staged through shared memory per 4-sample chunk) with
    L1-resident and L2-resident footprints, and the adjoint's float4 reductions with an
    L2-resident footprint. Rates are algorithmic bytes (8 corners per evaluation). Each figure: the best of 5 launches timed with CUDA events on the
    launching stream after one warm-up launch."""
    import ctypes

    from paper_2103_01954_gb300 import binding as B

    dev = torch.device("cuda", torch.cuda.current_device())
    M, steps = 16, 512
    out = {"access_pattern": "8 corners per lane and sample, 8x4-pixel warp tiles, lanes 1/4 voxel apart, "
                             "samples 2/3 voxel apart", "M": M, "footprint_l2_MB": 67}
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def timed(payload, dtype, n, mode, footprint, grad=None):
        acc = ctypes.c_int64(0)
        args = (ctypes.c_void_p(payload.data_ptr()) if payload is not None else None, dtype, n, M, mode, footprint,
                steps, ctypes.c_void_p(grad.data_ptr()) if grad is not None else None,
                ctypes.c_void_p(sink.data_ptr()), ctypes.byref(acc), stream)
        B.check(B.lib().mvp_gather_probe(*args), "mvp_gather_probe")
        best = None
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            B.check(B.lib().mvp_gather_probe(*args), "mvp_gather_probe")
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return acc.value, best

    n32 = 1024  # 1024 x 16^3 x 16 B = 67 MB (FP32); 2048 x 16^3 x 8 B = 67 MB (BF16)
    for name, tdt, dtype, vb in (("f32", torch.float32, B.MVP_F32, 16), ("bf16", torch.bfloat16, B.MVP_BF16, 8)):
        for mode, per, lay in ((0, 1, ""), (2, 2, "_xpair"), (3, 4, "_xyquad"), (4, 1, "_smem_staged")):
            n = n32 * 16 // (vb * per)  # the same 67 MB footprint for every layout
            payload = torch.rand((n, M, M, M, per, 4), device=dev).to(tdt)
            for fp, tag in ((0, "l1"), (1, "l2")):
                acc, ms = timed(payload, dtype, n, mode, fp)
                # algorithmic bytes: 8 corners of vb bytes per lane and sample
                out[f"gather_{name}{lay}_{tag}_GBps"] = round(acc * vb / (ms * 1e-3) / 1e9, 1)
            del payload
    g = torch.zeros((n32, M, M, M, 4), dtype=torch.float32, device=dev)
    acc, ms = timed(None, B.MVP_F32, n32, 1, 1, grad=g)
    out["scatter_f32x4_l2_Gupdates_s"] = round(acc / (ms * 1e-3) / 1e9, 2)
    # the same accesses at the residency the kernels get (4-warp blocks holding the march's
    # shared memory: 5 per SM for the march, 3 for the adjoint, as their launch bounds give)
    acc, ms = timed(None, B.MVP_F32, n32, 1 | (ADJOINT_BLOCKS_PER_SM << 8), 1, grad=g)
    out["scatter_f32x4_l2_at_adjoint_residency_Gupdates_s"] = round(acc / (ms * 1e-3) / 1e9, 2)
    del g
    for name, tdt, dtype, vb in (("f32", torch.float32, B.MVP_F32, 16), ("bf16", torch.bfloat16, B.MVP_BF16, 8)):
        n = n32 * 16 // vb
        payload = torch.rand((n, M, M, M, 4), device=dev).to(tdt)
        for fp, tag in ((0, "l1"), (1, "l2")):
            acc, ms = timed(payload, dtype, n, 0 | (MARCH_BLOCKS_PER_SM << 8), fp)
            out[f"gather_{name}_{tag}_at_march_residency_GBps"] = round(acc * vb / (ms * 1e-3) / 1e9, 1)
        del payload
    torch.cuda.empty_cache()
    return out


def _summary(variants, serving, probe):
    """Every part of the metric as flat scalars (the record keeps config's scalars)."""
    out = {}
    for key, name in (("fwd_bf16", "fwd_bf16_mrays_s"), ("fwd_f16", "fwd_f16_mrays_s"),
                      ("fwd_bwd_f32_512x32^3_4x512x512", "fwd_bwd_f32_512x32c_4x512x512_mrays_s"),
                      ("fwd_f32_512x32^3", "fwd_f32_512x32c_mrays_s"), ("fwd_f32_32768x8^3", "fwd_f32_32768x8c_mrays_s"),
                      ("fwd_bf16_32768x8^3", "fwd_bf16_32768x8c_mrays_s")):
        if isinstance(variants.get(key), dict) and "value" in variants[key]:
            out[name] = variants[key]["value"]
    fb = variants.get("fwd_bwd_f32_512x32^3_4x512x512")
    if fb:
        out["fwd_bwd_backward_ms"] = fb["backward_ms"]
        out["fwd_bwd_forward_ms"] = fb["forward_ms"]
        out["backward_scatter_frac"] = fb["backward_roofline"]["frac"]
        if fb["backward_roofline"].get("traffic_over_algorithmic") is not None:
            out["backward_dram_over_algorithmic"] = fb["backward_roofline"]["traffic_over_algorithmic"]
    for k in ("bf16_over_f32", "e2e_bf16_over_f32"):
        if k in variants:
            out[k] = variants[k]
    if isinstance(variants.get("fwd_bwd_f32_512x32^3_4x512x512"), dict):
        out["backward_scatter_frac_at_kernel_residency"] = \
            variants["fwd_bwd_f32_512x32^3_4x512x512"]["backward_roofline"]["frac_at_kernel_residency"]
    if isinstance(variants.get("fwd_bf16"), dict) and "gather_frac" in variants["fwd_bf16"]:
        out["fwd_bf16_gather_frac"] = variants["fwd_bf16"]["gather_frac"]
    for k, v in probe.items():
        if isinstance(v, (int, float)):
            out["probe_" + k] = v
    if serving:
        for rate, r in serving["rates"].items():
            tag = rate.replace(".0_req_per_s", "rps").replace("_req_per_s", "rps")
            out[f"serving_{tag}_requests"] = r["requests"]
            out[f"serving_{tag}_p50_ms"] = r["p50_ms"]
            out[f"serving_{tag}_p99_ms"] = r["p99_ms"]
            out[f"serving_{tag}_mrays_s"] = r["mrays_per_s"]
            out[f"serving_{tag}_one_at_a_time_f32_p50_ms"] = r["one_at_a_time_f32"]["p50_ms"]
            out[f"serving_{tag}_one_at_a_time_f32_p99_ms"] = r["one_at_a_time_f32"]["p99_ms"]
            out[f"serving_{tag}_one_at_a_time_f32_mrays_s"] = r["one_at_a_time_f32"]["mrays_per_s"]
            if "served_f32_payload" in r:
                out[f"serving_{tag}_served_f32_payload_mrays_s"] = r["served_f32_payload"]["mrays_per_s"]
    return out


def run_gpu(args):
    import torch

    import synthetic
    from paper_2103_01954_gb300 import torch_ops as T

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)
    peaks, peak_kind = _peaks()

    # headline: FP32 forward at paper scale; each rank renders its own seeded frame
    step, n_rays, info = _frame_runner(WORKLOAD, rank, "f32", False, torch, T, synthetic)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        durs = _time_steps(torch, step, args.steps, args.warmup, flush, time_march=True)
    info["ctx"].sync()
    ms, value = aggregate(float(np.mean(durs)), n_rays, ws, dev)
    march_ms = float(np.mean([a.elapsed_time(b) for a, b in info["ev"]["march"]]))
    # evaluations of one frame (the work count of the roofline)
    n_eval = int(T.raymarch_count(info["ctx"], info["prims"], info["bvh"], info["rs"]).sum().item())
    info["ctx"].sync()
    # rays whose opacity saturated (A = 1) in the frame
    saturated = float((info["out"][:, 3] >= 1.0).float().mean().item())

    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s (FMA = 2)
    ncu = _ncu_record("k_march_f32")
    probe = _gather_probe(torch, T)
    gather = GATHER_BYTES["f32"] * n_eval / (march_ms * 1e-3) / 1e9  # GB/s
    g_peak = probe["gather_f32_l1_GBps"]
    alu = FLOP_PER_EVAL * n_eval / (march_ms * 1e-3) / 1e12
    roofline = {"bound": "gather", "achieved": round(gather, 1), "peak": g_peak, "unit": "GB/s",
                "frac": round(gather / g_peak, 4), "traffic": ncu.get("dram_bytes_per_launch"),
                "peak_kind": "measured: mvp_gather_probe, the march's 8-corner FP32 gathers, L1-resident",
                "peak_l2_resident_GBps": probe["gather_f32_l2_GBps"],
                "frac_of_l2_resident": round(gather / probe["gather_f32_l2_GBps"], 4),
                "peak_at_kernel_residency_GBps": probe["gather_f32_l1_at_march_residency_GBps"],
                "frac_at_kernel_residency": round(gather / probe["gather_f32_l1_at_march_residency_GBps"], 4),
                "residency_note": "the same gathers at the march's 5 blocks of 4 warps per SM and its L1 size",
                "kernel": "k_march<f32>", "march_ms": round(march_ms, 4), "evaluations": n_eval,
                "bytes_per_evaluation": GATHER_BYTES["f32"],
                "l1_wavefront_frac": ncu.get("l1_wavefront_frac"),
                "alu_achieved_TFLOPs": round(alu, 3), "alu_peak_TFLOPs": round(fp32_peak, 2),
                "alu_frac": round(alu / fp32_peak, 4),
                "alu_peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock",
                "hbm_frac": (round(ncu["dram_bytes_per_launch"] / (march_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)
                             if ncu.get("dram_bytes_per_launch") and peaks.get("hbm_gbs") else None),
                "hbm_peak_GBps": peaks.get("hbm_gbs"), "hbm_peak_kind": peak_kind}
    # BVH: primitives + one-block sort (n <= 8192) or bounds, primitives and 4 radix
    # passes of 3 kernels; then hierarchy, refit; then the march and the next frame's
    # tile schedule
    launches_per_step = (2 if info["n_prims"] <= 8192 else 14) + 2 + 1 + 1
    result = {"metric": METRIC, "value": round(value, 3), "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; stands in for the paper's captures)",
              "config": {"workload": WORKLOAD, "primitives": 4096, "payload": "16^3 RGBA f32", "rays": n_rays,
                         "image": "667x1024", "dt": 0.005, "t_range": [1.0, 5.0], "samples_per_ray": 800,
                         "saturated_ray_fraction": round(saturated, 4),
                         "step": "BVH rebuild + traversal + march", "l2": "flushed (512 MiB write) before each step",
                         "stages_ms": {"bvh": round(ms - march_ms, 4), "march": round(march_ms, 4)},
                         "ms_per_step_median": round(float(np.median(durs)), 4),
                         "ms_per_step_p99": round(float(np.percentile(durs, 99)), 4),
                         "parallelism": f"replicas x{ws} (each rank its own frame)"},
              "roofline": roofline, "clocks": clk.summary(), "gpu_launches": launches_per_step * args.steps}
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
    if rank == 0 and not args.quick:
        result["e2e"] = _e2e(torch, T, info, max(20, args.steps), 3)
        result["e2e_rays_from_host"] = _e2e(torch, T, info, max(20, args.steps), 3, rays_from="host")
    del info, step
    torch.cuda.empty_cache()

    variants = {}
    if rank == 0 and not args.quick:
        for name, cfg, dtype, sched in (("fwd_bf16", WORKLOAD, "bf16", True), ("fwd_f16", WORKLOAD, "f16", True),
                                        ("fwd_f32_plain_tile_order", WORKLOAD, "f32", False),
                                        ("fwd_f32_512x32^3", "sweep_512x32^3_667x1024", "f32", True),
                                        ("fwd_f32_32768x8^3", "sweep_32768x8^3_667x1024", "f32", True),
                                        ("fwd_f32_32768x8^3_plain_tile_order", "sweep_32768x8^3_667x1024", "f32",
                                         False),
                                        ("fwd_f32_dt0.01", "paper_4096x16^3_667x1024_dt0.01", "f32", True),
                                        ("fwd_f32_dt0.0025", "paper_4096x16^3_667x1024_dt0.0025", "f32", True),
                                        ("fwd_bf16_32768x8^3", "sweep_32768x8^3_667x1024", "bf16", True)):
            st, nr, inf = _frame_runner(cfg, 0, dtype, False, torch, T, synthetic, schedule=sched)
            d = _time_steps(torch, st, args.steps, args.warmup, flush, time_march=True)
            inf["ctx"].sync()
            m = float(np.mean(d))
            mm = float(np.mean([a.elapsed_time(b) for a, b in inf["ev"]["march"]]))
            variants[name] = {"value": round(nr / (m * 1e-3) / 1e6, 3), "unit": "Mrays/s", "ms_per_step": round(m, 4),
                              "march_ms": round(mm, 4), "workload": cfg, "payload_dtype": dtype,
                              "tile_schedule": "by last frame's cost" if sched else "plain order"}
            if name == "fwd_bf16":
                # end to end with the payload streamed from the host as BF16 (half the bytes)
                e = _e2e(torch, T, inf, max(20, args.steps), 3, payload_dtype="bf16")
                variants["e2e_bf16"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in e.items()}
            del st, inf
            torch.cuda.empty_cache()
        variants["fwd_f32_sequential"] = _sequential_blend(torch, T, synthetic, args, flush)
        variants["orbiting_camera"] = _orbit(torch, T, synthetic, args, flush)
        st, nr, inf = _frame_runner("diff_512x32^3_4x512x512", 0, "f32", True, torch, T, synthetic)
        d = _time_steps(torch, st, args.steps, args.warmup, flush, time_march=True)
        inf["ctx"].sync()
        m = float(np.mean(d))
        bwd_ms = float(np.mean([a.elapsed_time(b) for a, b in inf["ev"]["bwd"]]))
        fwd_ms = float(np.mean([a.elapsed_time(b) for a, b in inf["ev"]["march"]]))
        e_diff = int(T.raymarch_count(inf["ctx"], inf["prims"], inf["bvh"], inf["rs"]).sum().item())
        inf["ctx"].sync()
        upd = 8 * e_diff / (bwd_ms * 1e-3) / 1e9  # float4 corner reductions per second (G)
        # the adjoint's algorithmic bytes: payload read, its gradient read and written, 72 B per ray
        alg = 3 * inf["n_prims"] * inf["M"] ** 3 * 16 + 72 * nr
        nb = _ncu_record("k_backward_grouped_f32")
        variants["fwd_bwd_f32_512x32^3_4x512x512"] = {
            "value": round(nr / (m * 1e-3) / 1e6, 3), "unit": "Mrays/s", "ms_per_step": round(m, 4),
            "forward_ms": round(fwd_ms, 4), "backward_ms": round(bwd_ms, 4),
            "workload": "diff_512x32^3_4x512x512", "step": "BVH + forward + L2 loss grad + backward (payload + pose)",
            "backward_roofline": {"bound": "scatter (float4 reductions)", "evaluations": e_diff,
                                  "achieved_Gupdates_s": round(upd, 2),
                                  "peak_Gupdates_s": probe["scatter_f32x4_l2_Gupdates_s"],
                                  "peak_kind": "measured: mvp_gather_probe mode 1, L2-resident footprint",
                                  "frac": round(upd / probe["scatter_f32x4_l2_Gupdates_s"], 4),
                                  "peak_at_kernel_residency_Gupdates_s":
                                      probe["scatter_f32x4_l2_at_adjoint_residency_Gupdates_s"],
                                  "frac_at_kernel_residency":
                                      round(upd / probe["scatter_f32x4_l2_at_adjoint_residency_Gupdates_s"], 4),
                                  "algorithmic_bytes": alg,
                                  "traffic": nb.get("dram_bytes_per_launch"),
                                  "traffic_over_algorithmic": (round(nb["dram_bytes_per_launch"] / alg, 3)
                                                               if nb.get("dram_bytes_per_launch") else None),
                                  "schedule": "primitive groups of a third of L2, replayed group after group"}}
        del st, inf
        torch.cuda.empty_cache()
        variants["fade_pack_bf16"] = _fade_pack(torch, T, synthetic, peaks)
        variants["pack"] = _pack(torch, T, synthetic, peaks)
        variants["vr_stereo_896x832"] = _vr_stereo(torch, T, synthetic, flush)
        variants["vr_stereo_view_dependent_896x832"] = _vr_stereo(torch, T, synthetic, flush, view_dependent=True)
        if variants.get("fwd_bf16"):
            variants["bf16_over_f32"] = round(variants["fwd_bf16"]["value"] / value, 3)
            gb = GATHER_BYTES["bf16"] * n_eval / (variants["fwd_bf16"]["march_ms"] * 1e-3) / 1e9
            variants["fwd_bf16"]["gather_GBps"] = round(gb, 1)
            variants["fwd_bf16"]["gather_frac"] = round(gb / probe["gather_bf16_l1_GBps"], 4)
        if variants.get("e2e_bf16") and result.get("e2e"):
            variants["e2e_bf16_over_f32"] = round(variants["e2e_bf16"]["value"] / result["e2e"]["value"], 3)
        result["variants"] = variants
        if args.serving_requests > 0:
            rates = [float(r) for r in args.serving_rates.split(",")]
            result["serving"] = _serving(torch, T, synthetic, rates, args.serving_requests)
            torch.cuda.empty_cache()
        if not args.no_cpu:
            result["cpu_baseline"] = _cpu_baseline(args.cpu_seconds)
        result["config"].update(_summary(variants, result.get("serving"), probe))
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


def run_reference(args):
    """The oracle on the host cores: each step renders a bounded seeded ray sample of
    the same workload; Mrays/s of the CPU path."""
    ws, rank = _dist()
    if rank != 0:
        return
    import oracle
    import synthetic

    oracle.build()
    scene, rays, _ = synthetic.make_config(WORKLOAD, 0)
    rng = np.random.default_rng(7)
    n = 2048
    cores = _host_threads()

    def step():
        sel = rng.choice(rays.n, n, replace=False)
        sub = synthetic.Rays(o=rays.o[sel], d=rays.d[sel], t_near=rays.t_near, t_far=rays.t_far, dt=rays.dt)
        oracle.render(scene, sub, n_threads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    sec = (time.perf_counter() - t0) / args.steps
    v = n / sec / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "Mrays/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rays_per_step": n, "sample": "seeded random pixels"},
            "cpu_baseline": {"value": round(v, 6), "unit": "Mrays/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} seeded random pixels of the 667x1024 frame per step"},
            "e2e": {"value": round(v, 6), "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_profile(args):
    """Render a few frames of one workload (for ncu captures): BVH build + march,
    and with --backward also the adjoint."""
    import torch

    import synthetic
    from paper_2103_01954_gb300 import torch_ops as T

    torch.cuda.set_device(0)
    step, _, info = _frame_runner(args.workload, 0, args.dtype, args.backward, torch, T, synthetic)
    for _ in range(args.frames):
        step()
    info["ctx"].sync()
    torch.cuda.synchronize()
    print(json.dumps({"profiled": args.workload, "frames": args.frames, "dtype": args.dtype,
                      "backward": args.backward}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--quick", action="store_true", help="headline figure only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serving-requests", type=int, default=2000, help="requests per arrival rate (0: skip)")
    ap.add_argument("--serving-rates", default="50,100,200,400,800,1200,1600", help="Poisson arrival rates, requests/s")
    ap.add_argument("--serving-only", action="store_true", help="run only the serving measurement")
    ap.add_argument("--profile", action="store_true", help="render --frames frames of --workload, no timing")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--frames", type=int, default=2)
    ap.add_argument("--backward", action="store_true")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
        return
    if args.serving_only:
        import torch

        import synthetic
        from paper_2103_01954_gb300 import torch_ops as T

        torch.cuda.set_device(0)
        rates = [float(r) for r in args.serving_rates.split(",")]
        print(json.dumps({"serving": _serving(torch, T, synthetic, rates, args.serving_requests)}))
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
