"""Continuous-batching request loop over the library's fr_server_* calls.

Requests arrive (Poisson, simulated clock), are admitted while the device has
free HBM for them (the driver's free-memory figure, or a fixed budget), are
planned into the server, and share its steps: each step is one launch of the
mapping kernel over a bounded number of voxels taken round-robin from every
admitted request, so a request that arrives while others are on the GPU is
mapped in the next launch alongside them.  Volumes and maps stay resident on
the device; finished requests are released, which frees memory for the next
admissions.  Reports throughput and latency percentiles.
"""
import collections
import ctypes as C
import time

import numpy as np

from . import _lib, _tune, check, fr_map_params_init


class Server:
    """Handle of an fr_server."""

    def __init__(self, device=0, max_radius=3, max_slots=512, tune=None):
        self.L = _lib.load()
        self.device = device
        h = C.c_void_p()
        check("fr_server_create", self.L.fr_server_create(device, max_radius, max_slots,
                                                          _tune(tune), C.byref(h)))
        self.handle = h

    def add(self, params, mask, image, out):
        """mask: torch uint8 (cpu or cuda); image int16 / out float32: cuda."""
        import torch
        if not isinstance(mask, torch.Tensor):
            mask = torch.from_numpy(mask)
        mask = mask.to(torch.uint8).contiguous()
        params.mask_on_device = 1 if mask.is_cuda else 0
        params.device = self.device
        rid = C.c_int64()
        check("fr_server_add", self.L.fr_server_add(
            self.handle, C.byref(params), C.c_void_p(mask.data_ptr()),
            C.c_void_p(image.data_ptr()), C.c_void_p(out.data_ptr()), C.byref(rid)))
        return rid.value

    def step(self, voxel_budget):
        n = C.c_int32()
        check("fr_server_step", self.L.fr_server_step(self.handle, int(voxel_budget), C.byref(n)))
        return n.value

    def poll(self, wait=False, cap=4096):
        ids = (C.c_int64 * cap)()
        sts = (C.c_int32 * cap)()
        n = C.c_int32()
        check("fr_server_poll", self.L.fr_server_poll(self.handle, 1 if wait else 0, ids, sts,
                                                      cap, C.byref(n)))
        return [(ids[k], sts[k]) for k in range(n.value)]

    def release(self, rid):
        check("fr_server_release", self.L.fr_server_release(self.handle, int(rid)))

    def query(self):
        a, f, b = C.c_int32(), C.c_int32(), C.c_size_t()
        check("fr_server_query", self.L.fr_server_query(self.handle, C.byref(a), C.byref(f),
                                                        C.byref(b)))
        return a.value, f.value, b.value

    def close(self):
        if getattr(self, "handle", None):
            self.L.fr_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def request_bytes(shape, n_voi, n_rows, brick=(8, 4, 4), voxels_per_item=16):
    """Device bytes one admitted request holds: output maps, packed volume,
    VOI list and brick-ordered columns, and the plan's temporaries (mask copy,
    row and brick counters)."""
    nz, ny, nx = shape
    px = (nx + 3) // 4 * 4
    nb = -(-nx // brick[0]) * -(-ny // brick[1]) * -(-nz // brick[2])
    return (4 * n_rows * n_voi + 4 * px * ny * nz + 8 * n_voi + nz * ny * nx + 8 * ny * nz
            + 12 * nb + 24 * (n_voi // voxels_per_item + nb) + 4096)


def serve(requests, images, rate, *, seed=0, voxel_budget=65536, hbm_reserve=4 << 30,
          hbm_budget=None, device=0, max_radius=3, keep_outputs=False, tune=None,
          time_limit=None, drain_dir=None, drain_codec="gzip", drain_workers=2,
          admit_per_step=6, max_active=256):
    """Run the request stream; returns a dict of statistics (and the outputs
    by request index when keep_outputs).

    requests: dicts with mask (numpy uint8), shape, radius, disc (parameter
    overrides), n_voi, and either image_key (a key of `images`, device int16
    tensors) or the shape used as the key.  rate: mean arrivals per second.
    hbm_budget: admit against this many bytes instead of the driver's free
    memory (the in-use figure is the sum of admitted estimates).
    drain_dir: write each finished request to <drain_dir>/request_<i>.h5
    (fr_h5_write_maps) on host worker threads, off the GPU loop; the maps are
    copied to the host first, so the request's device memory is released at
    once.  Latencies count up to the device result, not the file.
    admit_per_step: requests planned per loop turn while others are on the
    GPU, so planning never leaves the two steps in flight without a
    successor for long.  max_active: admitted requests at most (the
    server's slots); beyond it arrivals wait in the queue, which counts in
    their latency."""
    import torch
    n = len(requests)
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n)) if rate > 0 else np.zeros(n)
    srv = Server(device, max_radius=max_radius, max_slots=max_active, tune=tune)
    pending = collections.deque(range(n))
    active = {}
    latency = np.full(n, np.nan)
    admit_at = np.full(n, np.nan)
    outputs = {}
    in_use = 0
    peak_in_use = 0
    done = 0
    feats = 93  # the default selection: the benchmark maps
    steps = 0
    drainer = None
    drained = []
    if drain_dir is not None:
        import concurrent.futures as cf
        import os
        os.makedirs(drain_dir, exist_ok=True)
        drainer = cf.ThreadPoolExecutor(max_workers=drain_workers)

    def drain(i, params, maps):
        from . import fr_h5_write_maps
        import os
        rq = requests[i]
        img = images[rq.get("image_key", rq["shape"])]
        mask = rq["mask"]
        vox = np.flatnonzero(np.asarray(mask).reshape(-1)).astype(np.int32)
        path = os.path.join(drain_dir, "request_%d.h5" % i)
        t = time.perf_counter()
        fr_h5_write_maps(path, params, img, mask, maps, vox, codec=drain_codec,
                         source_id="request %d" % i, threads=4)
        return path, time.perf_counter() - t

    t0 = time.perf_counter()
    while done < n:
        now = time.perf_counter() - t0
        if time_limit is not None and now > time_limit:
            break
        # admission: arrived requests, in order, while memory and slots allow
        admitted = 0
        while (pending and arrivals[pending[0]] <= now and len(active) < max_active and
               (admitted < admit_per_step or not active)):
            i = pending[0]
            rq = requests[i]
            est = request_bytes(rq["shape"], rq["n_voi"], feats)
            if hbm_budget is not None:
                room = hbm_budget - in_use
            else:
                room = torch.cuda.mem_get_info(device)[0] - hbm_reserve
            if est > room and active:
                break  # wait for finished requests to free memory
            nz, ny, nx = rq["shape"]
            p = fr_map_params_init(nx, ny, nz, kernel_radius=rq["radius"], **rq["disc"])
            out = torch.empty((feats, rq["n_voi"]), dtype=torch.float32, device="cuda:%d" % device)
            img = images[rq.get("image_key", rq["shape"])]
            rid = srv.add(p, rq["mask"], img, out)
            active[rid] = (i, out, est, p)
            admit_at[i] = time.perf_counter() - t0
            in_use += est
            peak_in_use = max(peak_in_use, in_use)
            pending.popleft()
            admitted += 1
        if active:
            srv.step(voxel_budget)
            steps += 1
            finished = srv.poll(wait=False)
            if not finished and not (pending and arrivals[pending[0]] <= now):
                finished = srv.poll(wait=True)
            for rid, st in finished:
                i, out, est, p = active.pop(rid)
                if st != 0:
                    raise RuntimeError("request %d finished with status %d" % (i, st))
                latency[i] = time.perf_counter() - t0 - arrivals[i]
                if keep_outputs:
                    outputs[i] = out
                if drainer is not None:
                    drained.append(drainer.submit(drain, i, p, out.cpu().numpy()))
                srv.release(rid)
                in_use -= est
                done += 1
        elif pending:
            time.sleep(max(0.0, min(0.01, arrivals[pending[0]] - now)))
    makespan = time.perf_counter() - t0
    srv.close()
    drain_files = None
    if drainer is not None:
        drain_files = [f.result() for f in drained]
        drainer.shutdown()
    ok = ~np.isnan(latency)
    vf = float(sum(requests[i]["n_voi"] for i in range(n) if ok[i]) * feats)
    stats = {
        "requests": int(ok.sum()), "rate": rate, "makespan_s": makespan, "steps": steps,
        "throughput": vf / makespan if makespan > 0 else 0.0,
        "p50_s": float(np.percentile(latency[ok], 50)) if ok.any() else None,
        "p99_s": float(np.percentile(latency[ok], 99)) if ok.any() else None,
        "mean_s": float(np.mean(latency[ok])) if ok.any() else None,
        "peak_admitted_bytes": int(peak_in_use),
        "queue_wait_p99_s": float(np.nanpercentile(admit_at - arrivals, 99)) if ok.any() else None,
    }
    if keep_outputs:
        stats["outputs"] = outputs
    if drain_files is not None:
        stats["drained"] = drain_files
    return stats
