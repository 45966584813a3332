#!/usr/bin/env python3
"""Benchmark of the fused two-component Shan-Chen D3Q19 step.

Workload (default): the fully resolved drainage sample, 192^3 lattice, 300
non-overlapping spheres with radii U[10, 14] placed by seeded random
sequential addition, inlet reservoir layer z = 0, three membrane layers and
the outlet reservoir layer at the top, FP32 populations.  One bench step is
one time step of the whole domain (one launch of the fused step kernel).

Printed JSON line (rank 0):
  value      fluid-cell updates per second (MLUPS) with the state resident in
             HBM, CUDA events around exactly --steps launches, max over ranks;
  roofline   the step kernel against HBM bandwidth: algorithmic bytes
             (2 x 19 populations read + written per fluid cell) / mean launch time;
  e2e        the same metric through the public C ABI from host data: domain
             creation from the host sphere list, then per step
             set_pressure_bc + 100 time steps + a measurement read back;
  cpu_baseline  the FP64 oracle on a bounded crop of the same sample;
  throats    pore throats per second on 1024 Delaunay throats of the sample
             packing (boxes 24^3..64^3): the plain per-throat loop (create,
             ladder of set_pressure_bc + steps + measure, destroy) on a strided
             subset, the batch (cell-list form, with the tile and persistent
             forms beside it), and the surrogate (trained on six other packings)
             with batched-LBM fallback where the ensemble spread exceeds 2 % (and
             5 %), with the surrogate's p_c^e error against the batched LBM.
--impl reference times that oracle alone (the method has no other reference
implementation): rank 0 only.  --drainage runs the sample's full drainage;
--throat-batch FORM times one 1024-throat batch in one form.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

POP_STORAGE = {0: "FP32 populations", 1: "FP16 population deviations", 2: "BF16 population deviations"}
METRIC = "D3Q19 2-comp Shan-Chen MLUPS & % HBM peak; pore throats/s vs plain"
FALLBACK_HBM_GBS = 6800.0
E2E_SUBSTEPS = 100


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-throats", action="store_true")
    ap.add_argument("--precision", type=int, choices=[0, 1, 2], default=0,
                    help="population storage: 0 FP32 (the benchmark), 1 FP16 / 2 BF16 deviations")
    ap.add_argument("--drainage", action="store_true",
                    help="instead of the benchmark: the full drainage of the sample (20 increments x --pn-steps "
                         "steps), one JSON line with the p_c - S_w curve")
    ap.add_argument("--no-tune", action="store_true", help="time the default kernel instead of the autotuned one")
    ap.add_argument("--pore-network", action="store_true",
                    help="drainage of the sample by the pore network (throat entry pressures from the batched "
                         "LBM and the incircle estimate) next to the full LBM drainage, one JSON line")
    ap.add_argument("--pn-steps", default="5000",
                    help="full-LBM steps per increment for --pore-network (a comma list runs the full LBM at each; "
                         "the network is compared with the last)")
    ap.add_argument("--throat-convergence", action="store_true",
                    help="p_c^e of 64 throats against the steps per pressure increment (100 .. 4000), one JSON line")
    ap.add_argument("--surrogate-config5", action="store_true",
                    help="the throat surrogate at configuration 5's size (20 k training throats, 1e5 inference "
                         "throats of 2000-sphere packings, LBM fallback at 2 %% spread), one JSON line")
    ap.add_argument("--train-throats", type=int, default=20000,
                    help="--surrogate-config5: LBM training throats (whole packings until reached)")
    ap.add_argument("--judge", type=int, default=2000,
                    help="--surrogate-config5: inference throats the LBM judges (seeded random subset)")
    ap.add_argument("--refine", type=int, default=1,
                    help="--surrogate-config5: entry pressures refined to 1/N of a ladder step "
                         "(lbm_run_throat_batch_refined) for the labels and the judge; 1 = the ladder's own")
    ap.add_argument("--shape", default="",
                    help="fixed step kernel shape instead of tuning: tma:LZ, split, staged:BY:LZ:LEAD, "
                         "staged2:BY:LZ:2 or push:SHAPE:LZ[:PREFETCH[:ORDER]] (SHAPE an lbm_set_push_shape index)")
    ap.add_argument("--throat-steps", type=int, default=100,
                    help="time steps per pressure increment of the throat ladder (32 increments)")
    ap.add_argument("--throat-batch", default="",
                    help="instead of the benchmark: one batch of the 1024 held-out throats in the given form "
                         "(cells, tiles, persistent, march or march:THREADS:PLANES; 32 increments), and the same "
                         "batch with no time steps (the set-up cost)")
    ap.add_argument("--throat-count", type=int, default=1024,
                    help="with --throat-batch: every (1024 // count)-th throat of the packing (profiling captures)")
    ap.add_argument("--size", type=int, default=192,
                    help="box edge of the drainage sample (192 = the benchmark workload; smaller edges "
                         "scale the sphere count with the volume, for profiling captures)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest value over all ranks (the job ends when its slowest rank
    does); the value itself without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds_local: float, world: int, dist=None, device="cpu") -> float:
    """Units per second of the whole job: every rank processed units_per_rank
    (replicas, weak scaling) in at most the slowest rank's time."""
    return world * units_per_rank / max_over_ranks(seconds_local, dist, device)


def sample_geometry(edge: int = 192):
    import workloads as W
    return W.sample_spheres(edge), (edge, edge, edge)


def update_bytes(mask):
    """Algorithmic bytes of one step: 19 populations x 4 B read + 4 B written
    per component present at each non-solid cell (membrane cells carry only the
    wetting component)."""
    solid = (mask & 1) != 0
    memb = (mask & 4) != 0
    n_w = int((~solid).sum())
    n_nw = int((~solid & ~memb).sum())
    return n_w, n_w * 152 + n_nw * 152


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm_gb_s"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# the sources each step kernel is compiled from: a traffic record holds while they are unchanged
KERNEL_SOURCES = {
    "sc_step_kernel": ("lbm_step.cu", "lbm_step_core.cuh", "lbm_device.cuh", "lbm_internal.h"),
    "sc_step_tma_kernel": ("lbm_step_tma.cu", "lbm_step_core.cuh", "lbm_device.cuh", "lbm_internal.h"),
    "sc_step_push_kernel": ("lbm_step_push.cu", "lbm_push_tma.cuh", "lbm_step_core.cuh", "lbm_device.cuh",
                            "lbm_internal.h"),
    "sc_step16_push_kernel": ("lbm_step16_push.cuh", "lbm_step16_push.cu", "lbm_step16_push_bf16.cu",
                              "lbm_pair16.cuh", "lbm_push_tma.cuh", "lbm_step_core.cuh", "lbm_device.cuh",
                              "lbm_internal.h"),
}


def kernel_hash(kernel_name="sc_step_kernel"):
    key = next((k for k in ("sc_step_tma_kernel", "sc_step_push_kernel", "sc_step16_push_kernel")
                if kernel_name.startswith(k)),
               "sc_step_kernel")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[key]:
        h.update(open(os.path.join(ROOT, "paper_1906_04722_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(kernel_name):
    """DRAM bytes per launch of the given step kernel on the 192^3 sample from
    the committed ncu summary, valid only while that kernel's sources are
    unchanged (the caller asks only for that workload)."""
    p = os.path.join(ROOT, "profiles", "sc_step_sample192_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        k = d.get("kernels", {}).get(kernel_name)
        if k and k.get("kernel_hash") == kernel_hash(kernel_name):
            return float(k["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.idx = gpu_index

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


class OracleCrop:
    """The FP64 oracle on a 64^3 crop of the 192^3 sample (same packing shifted
    so that x, y in [64, 128) of the sample fill the crop, reservoir layer at the
    inlet end, membrane and outlet at the other), timed on the host's cores."""

    def __init__(self):
        import oracle
        import workloads as W
        spheres, _ = sample_geometry()
        self.shape = (64, 64, 64)
        sh = spheres.copy()
        sh[:, :3] -= np.array([64.0, 64.0, 0.0])
        self.oracle = oracle
        self.mask = oracle.voxelise(self.shape, sh, reservoirs=True, membrane_layers=3)
        self.cfg = oracle.Config(shape=self.shape, tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS,
                                 rho_in=(W.RHO_MINOR, W.RHO_MAJOR), rho_out=(W.RHO_MAJOR, W.RHO_MINOR))
        self.f = oracle.init(self.cfg, self.mask, W.initial_densities(self.shape))
        self.n_update = int(((self.mask & 1) == 0).sum())
        self.cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))

    def time_steps(self, n):
        t0 = time.perf_counter()
        self.oracle.step(self.cfg, self.mask, self.f, n)
        return time.perf_counter() - t0

    def sample_text(self, steps):
        return (f"64^3 crop of the 192^3 sample (x, y in [64, 128)), {steps} FP64 oracle steps, "
                f"{self.n_update} fluid cells per step")


def cpu_baseline():
    """About 15 s of oracle work on the crop."""
    oc = OracleCrop()
    oc.time_steps(1)
    dt1 = oc.time_steps(2) / 2
    steps = max(1, min(4000, int(15.0 / max(dt1, 1e-3))))
    dt = oc.time_steps(steps)
    return {"value": oc.n_update * steps / dt / 1e6, "unit": "MLUPS", "cores": oc.cores, "kind": "oracle",
            "sample": oc.sample_text(steps)}


def throat_bench(lbm, W, n_steps, rank, world, sync, tmax, gather=None):
    """Throats per second: plain loop vs batched vs surrogate with fallback.

    The ladder is 32 increments of the nw reservoir density (2.0 + 0.02 i) with
    n_steps time steps each, for every arm.  The surrogate is trained first on
    six other seeded packings (its cost is reported, not counted in throats/s:
    it is paid once for all throats of a network).  Every rank works on its own
    held-out packing; tmax(t) is the maximum of t over ranks, and the rates
    are whole-job: world x throats per rank / that maximum."""
    from paper_1906_04722_gb300 import surrogate as S

    params = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                             rho_minor=W.RHO_MINOR)
    theta = S.contact_angle_estimate(W.G_ADS[0], W.G_ADS[1], W.G_COHESION, W.RHO_MAJOR, W.RHO_MINOR)
    ladder = [W.RHO_MAJOR + 0.02 * i for i in range(32)]
    out = {"workload": "1024 throats (facets of the regular triangulation, longest centre distance < 64) of a "
                       f"300-sphere 192^3 RSA packing, 32 increments x {n_steps} steps", "unit": "throats/s"}
    # training set from six other packings
    t0 = time.perf_counter()
    tris, ress, rowss = [], [], []
    for seed in range(10 + 6 * rank, 16 + 6 * rank):
        tri = lbm.packing_throat_sample(W.sample_spheres(192, seed=100 + seed), 1024, seed=100 + seed)
        res, rows = lbm.lbm_run_throat_batch(tri, params, ladder, n_steps, W.RHO_MAJOR)
        tris.append(tri)
        ress += res
        rowss += rows
    t_gen = time.perf_counter() - t0
    sur = S.ThroatSurrogate(n_incr=len(ladder), theta=theta, n_members=5, seed=1)
    t0 = time.perf_counter()
    losses, used = sur.fit(np.concatenate(tris), ress, rowss, epochs=300, batch=256, lr=1e-3, seed=2)
    t_train = time.perf_counter() - t0
    out["surrogate_training"] = {"throats": int(used), "lbm_s": t_gen, "train_s": t_train,
                                 "loss_first_last": [float(losses[:, 0].mean()), float(losses[:, -1].mean())]}

    tri = lbm.packing_throat_sample(W.sample_spheres(192, seed=3 + 1000 * rank), 1024, seed=3 + 1000 * rank)
    n = len(tri)
    # batched
    sync()
    t0 = time.perf_counter()
    res_ref, _ = lbm.lbm_run_throat_batch(tri, params, ladder, n_steps, W.RHO_MAJOR)
    sync()
    t_batch = tmax(time.perf_counter() - t0)
    truth = np.array([r["p_ce"] for r in res_ref])
    out["batched"] = world * n / t_batch
    # the analytic estimates Sec. 1 cites, on the same throats (sigma from
    # Laplace's law on the GPU, the contact angle of the adhesion estimate)
    sigma, _ = laplace_sigma(lbm, W)
    cos_t = math.cos(theta)
    fin = np.isfinite(truth)
    out["baselines"] = {"sigma": sigma, "cos_theta": cos_t}
    for name, est in (("incircle", lbm.lbm_throat_pce_incircle(tri, sigma, cos_t)),
                      ("msp", lbm.lbm_throat_pce_msp(tri, sigma, cos_t))):
        ok = fin & np.isfinite(est)
        rel = np.abs(est[ok] - truth[ok]) / np.abs(truth[ok])
        out["baselines"][name] = {"median_ratio_to_lbm": float(np.median(est[ok] / truth[ok])),
                                  "rel_err_median": float(np.median(rel)), "rel_err_p90": float(np.percentile(rel, 90))}
    out["batch_form"] = ("cell list: compact storage of every non-solid cell, a density launch and a push-streaming "
                         "step launch per time step")
    # the same batch in the other two forms, for context
    out["other_forms"] = {}
    agree = True
    for form, name in ((lbm.BATCH_MARCH, "march"), (lbm.BATCH_PER_STEP, "tiles_per_step"),
                       (lbm.BATCH_PERSISTENT, "persistent")):
        sync()
        t0 = time.perf_counter()
        res_f, _ = lbm.lbm_run_throat_batch(tri, params, ladder, n_steps, W.RHO_MAJOR, form=form)
        sync()
        out["other_forms"][name] = world * n / tmax(time.perf_counter() - t0)
        agree &= bool(np.array_equal(truth, np.array([r["p_ce"] for r in res_f]), equal_nan=True))
    out["forms_agree"] = agree
    if world > 1 and gather is not None:
        # one throat list over all ranks: LPT shards on the non-solid cells of
        # each box, results gathered back into the list's order
        shared = lbm.packing_throat_sample(W.sample_spheres(192, seed=3), 1024, seed=3)
        sync()
        t0 = time.perf_counter()
        res_s, _ = lbm.run_throat_batch_sharded(shared, params, ladder, n_steps, W.RHO_MAJOR, rank, world, gather)
        sync()
        out["sharded_one_list"] = {"throats": len(shared), "ranks": world,
                                   "throats_per_s": len(shared) / tmax(time.perf_counter() - t0),
                                   "all_gathered": all(r is not None for r in res_s)}
    # plain per-throat loop on every 16th throat
    sub = tri[::16]
    per = []
    sync()
    t0 = time.perf_counter()
    for th in sub:
        t1 = time.perf_counter()
        mask, probe = lbm.lbm_throat_geometry(th)
        d = lbm.Domain(params, mask=mask)
        d.drainage(ladder, n_steps, W.RHO_MAJOR, probe)
        d.close()
        per.append(time.perf_counter() - t1)
    sync()
    t_plain = tmax(time.perf_counter() - t0)
    out["plain"] = world * len(sub) / t_plain
    out["plain_sample"] = f"{len(sub)} throats (every 16th)"
    out["plain_seconds_per_throat"] = {"p10": float(np.percentile(per, 10)), "median": float(np.median(per)),
                                       "p90": float(np.percentile(per, 90)), "max": float(np.max(per))}
    out["batched_vs_plain"] = out["batched"] / out["plain"]
    ok = np.isfinite(truth)
    for tol in (0.02, 0.05):
        sur.spread_tol = tol
        sync()
        t0 = time.perf_counter()
        pce, fell, _, _ = sur.predict_with_fallback(tri, params, ladder, n_steps, W.RHO_MAJOR)
        sync()
        dt = tmax(time.perf_counter() - t0)
        ans = ok & ~fell
        err = np.abs(pce[ans] - truth[ans]) / truth[ans]
        out[f"surrogate_spread_{int(tol * 100)}pct"] = {
            "value": world * n / dt, "vs_plain": world * n / dt / out["plain"], "fallback_fraction": float(fell.mean()),
            "pce_rel_err_answered_median": float(np.median(err)) if err.size else None,
            "pce_rel_err_answered_p90": float(np.percentile(err, 90)) if err.size else None}
    sur.close()
    return out


def run_reference(args, rank, world):
    """The oracle itself as the reference arm, on the host cores, rank 0 only."""
    if rank != 0:
        return 0
    oc = OracleCrop()
    for _ in range(args.warmup):
        oc.time_steps(1)
    steps = max(1, args.steps)
    t_all = sum(oc.time_steps(1) for _ in range(steps))
    value = oc.n_update * steps / t_all / 1e6
    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus, "steps": steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_all / steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": "sample192, 64^3 crop (FP64 oracle on host cores)", "global_batch": 1,
                      "seq_len": 0, "parallelism": "host OpenMP threads"},
           "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oc.cores, "kind": "oracle",
                            "sample": oc.sample_text(steps)},
           "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_ours(args, rank, world, local):
    import torch
    import paper_1906_04722_gb300 as lbm
    import workloads as W

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device for --impl ours")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    spheres, box = sample_geometry(args.size)
    params = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                             rho_minor=W.RHO_MINOR, reservoirs=True, membrane_layers=3, precision=args.precision)
    stream = torch.cuda.Stream()
    dom = lbm.Domain(params, spheres, box, stream=ctypes.c_void_p(stream.cuda_stream))
    mask = dom.mask()
    n_upd, bytes_per_step = update_bytes(mask)
    if args.precision:
        # 16-bit storage: 19 pair words read + written and the density pair read
        # + written per non-solid cell
        bytes_per_step = n_upd * (19 * 4 * 2 + 8 + 8)
    # one population buffer: 19 slots of (w, nw) pairs of 4-byte floats or of a
    # 4-byte word of two 16-bit deviations per cell
    pop_buffer_gb = 19 * (8 if args.precision == 0 else 4) * box[0] * box[1] * box[2] / 1e9
    dom.set_pressure_bc(2.1, W.RHO_MAJOR)
    # the library's autotuner picks the step kernel and its launch shape on this
    # domain (state restored afterwards); untimed
    if args.shape:
        f = args.shape.split(":")
        if f[0] == "push":  # push:shape:lz[:prefetch planes]
            sh = int(f[1])
            table = lbm.PUSH16_SHAPE_TABLE if args.precision else lbm.PUSH_SHAPE_TABLE
            tuned = {"kind": "push", "shape": sh, "by": table[sh][0], "lz": int(f[2]),
                     "lead": table[sh][1], "prefetch": int(f[3]) if len(f) > 3 else 0,
                     "order": int(f[4]) if len(f) > 4 else 0}
        else:
            tuned = ({"kind": "tma", "lz": int(f[1])} if f[0] == "tma" else {"kind": "split"} if f[0] == "split" else
                     {"kind": f[0], "by": int(f[1]), "lz": int(f[2]), "lead": int(f[3])})
    else:
        tuned = dom.autotune(trial_steps=20) if not args.no_tune else None

    def apply_tuned(d):
        if tuned is None:
            return
        if tuned["kind"] == "push":
            d.set_push_shape(tuned["shape"], tuned["lz"])
            d.set_push_prefetch(tuned.get("prefetch", 0))
            d.set_push_order(tuned.get("order", 0))
        elif tuned["kind"] == "tma":
            d.set_step_kernel(lbm.KERNEL_TMA, tuned["lz"])
        elif tuned["kind"] == "split":
            d.set_step_kernel(lbm.KERNEL_SPLIT)
        elif tuned["kind"] == "staged2":
            d.set_tile(tuned["by"], tuned["lz"], 2)
            d.set_step_kernel(lbm.KERNEL_STAGED2, tuned["lz"])
        else:
            d.set_tile(tuned["by"], tuned["lz"], tuned["lead"])

    apply_tuned(dom)

    kind, _ = dom.step_kernel()
    h2 = "half2" if args.precision == 1 else "bfloat162"
    if args.precision and kind == lbm.KERNEL_PUSH:
        rows, stages, ctas = lbm.PUSH16_SHAPE_TABLE[tuned["shape"]][:3]
        kernel_name = "sc_step16_push_kernel<%s,%d,%d,%d>" % (h2, rows, stages, ctas)
    elif args.precision:
        by, _, lead = lbm.lbm_get_tile(dom.h)
        kernel_name = "sc_step16_kernel<%s,%d,%d>" % (h2, by, lead)
    elif kind == lbm.KERNEL_PUSH:
        rows, stages, ctas, resident = lbm.PUSH_SHAPE_TABLE[tuned["shape"]]
        kernel_name = "sc_step_push_kernel<%d,%d,%d,%s,%s>" % (
            rows, stages, ctas, "true" if tuple(W.TAU) == (1.0, 1.0) else "false", "true" if resident else "false")
    elif kind == lbm.KERNEL_TMA:
        kernel_name = "sc_step_tma_kernel"
    elif kind == lbm.KERNEL_SPLIT:
        kernel_name = "density_pair_kernel + sc_step_split_kernel (one step)"
    elif kind == lbm.KERNEL_STAGED2:
        kernel_name = "sc_step2_kernel<%d,2>" % lbm.lbm_get_tile(dom.h)[0]
    else:
        by, _, lead = lbm.lbm_get_tile(dom.h)
        kernel_name = ("sc_step_kernel<%d,%d>" if lead >= 2 else "sc_step_dp_kernel<%d,%d>") % (by, lead)
    dom.step(args.warmup)
    torch.cuda.synchronize()

    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        evs[0].record(stream)
        for i in range(args.steps):
            dom.step(1)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
    barrier()
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    value = whole_job_rate(n_upd * args.steps, total_ms / 1e3, world) / 1e6
    mean_ms = float(np.mean(per))
    peak, peak_kind = read_peaks()
    achieved = bytes_per_step / (mean_ms / 1e3) / 1e9
    m = dom.measure()
    dom.close()

    # end to end through the C ABI from host data
    e2e_val = None
    h2d = d2h = 0
    if args.e2e_steps > 0:
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2 = lbm.Domain(params, spheres, box)
        apply_tuned(d2)
        ladder = [W.RHO_MAJOR + 0.005 * i for i in range(args.e2e_steps)]
        for rin in ladder:
            d2.set_pressure_bc(rin, W.RHO_MAJOR)
            d2.step(E2E_SUBSTEPS)
            d2.measure()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        d2.close()
        N = box[0] * box[1] * box[2]
        e2e_val = world * n_upd * E2E_SUBSTEPS * args.e2e_steps / dt / 1e6
        h2d = int((N + spheres.nbytes) / args.e2e_steps) + 16  # mask (voxelised on the host), spheres, BC values
        d2h = 16 * 8

    clocks = clk.summary()

    def tmax(v):
        return max_over_ranks(v, dist, "cuda")

    def sync():
        torch.cuda.synchronize()
        barrier()

    def gather(obj):
        got = [None] * world
        dist.all_gather_object(got, obj)
        return got

    throats = None if args.no_throats else throat_bench(lbm, W, args.throat_steps, rank, world, sync, tmax,
                                                        gather if dist is not None else None)
    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": {0: "f32", 1: "f16 deviations, f32 math", 2: "bf16 deviations, f32 math"}[args.precision],
           "data": "synthetic",
           "config": {"workload": f"sample{args.size}: {args.size}^3, {len(spheres)} RSA spheres r~U[10,14], "
                                  f"reservoirs + 3 membrane layers, {POP_STORAGE[args.precision]}, one fused step per launch",
                      "fluid_cells": n_upd, "global_batch": world, "seq_len": 0,
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "l2": "inputs larger than L2 (2 x %.2f GB population buffers)" % pop_buffer_gb,
                      "step_kernel": tuned if tuned is not None else "default"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": read_traffic(kernel_name) if args.size == 192 else None, "peak_kind": peak_kind,
                        "kernel": kernel_name, "algorithmic_bytes_per_launch": bytes_per_step},
           "gpu_launches": args.steps * (2 if kind == lbm.KERNEL_SPLIT and not args.precision else 1),
           "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "step": f"set_pressure_bc + {E2E_SUBSTEPS} time steps + lbm_measure; domain creation "
                           "from the host sphere list inside the timed region"},
           "check": {"S_w": m["S_w"], "p_c_res": m["p_c_res"], "mass": m["mass"]}}
    if clocks:
        out["clocks"] = clocks
    if throats is not None:
        out["throats"] = throats
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline()
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_drainage(args):
    """The fully resolved drainage of the sample: the non-wetting reservoir
    density raised by 0.02 per increment (20 increments), --pn-steps steps each
    (a comma list runs the ladder once per entry, from the same start), the
    observables of lbm_measure after every increment (Sec. 2.2.2, Sec. 3.1)."""
    import torch
    import paper_1906_04722_gb300 as lbm
    import workloads as W

    spheres, box = sample_geometry(args.size)
    params = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                             rho_minor=W.RHO_MINOR, reservoirs=True, membrane_layers=3)
    ladder = [W.RHO_MAJOR + 0.02 * i for i in range(20)]
    # invasion probe: the centre of the last fluid layer before the membrane
    probe = (box[0] // 2, box[1] // 2, box[2] - 6)
    runs = {}
    for ns in [int(x) for x in str(args.pn_steps).split(",")]:
        dom = lbm.Domain(params, spheres, box)
        tuned = dom.autotune(trial_steps=10)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = dom.drainage(ladder, ns, W.RHO_MAJOR, probe)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dom.close()
        rows = [{k: r[k] for k in ("rho_in_nw", "p_c", "p_c_res", "S_w", "n_interface", "phi_probe")}
                for r in out["rows"]]
        runs[str(ns)] = {"step_kernel": tuned, "seconds": dt, "steps_per_s": 20 * ns / dt,
                         "invaded_at": out["invaded_at"], "p_ce": out["p_ce"], "rows": rows}
    print(json.dumps({"workload": f"sample{args.size} drainage, 20 increments of +0.02, steps per increment: "
                                  f"{args.pn_steps}", "runs": runs}))
    return 0


def laplace_sigma(lbm, W, edge=48, radii=(8.0, 12.0), steps=4000):
    """Interfacial tension of the model from Laplace's law on the GPU: static
    non-wetting drops of two radii in a periodic box, dp = p_nw - p_w of the bulk
    phases (Eq. 5), R from the drop's volume; sigma = dp R / 2 averaged."""
    params = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=(0.0, 0.0), rho_major=W.RHO_MAJOR,
                             rho_minor=W.RHO_MINOR, periodic=(1, 1, 1))
    shape = (edge, edge, edge)
    out = []
    for R0 in radii:
        with lbm.Domain(params, None, shape) as d:
            d.set_densities(W.droplet_densities(shape, (edge / 2, edge / 2, edge / 2), R0, seed=1, noise=0.0))
            d.step(steps)
            m = d.measure()
        vol = m["n_fluid"] - m["n_w"]
        R = (3.0 * vol / (4.0 * math.pi)) ** (1.0 / 3.0)
        out.append((R, m["p_nw"] - m["p_w"]))
    return float(np.mean([dp * R / 2.0 for R, dp in out])), out


def run_pore_network(args):
    """Row f1: drainage of the 192^3 sample by the pore network (Sec. 2.2.1 -
    2.2.2, Sec. 3.1.1) next to the fully resolved LBM drainage.  The network is
    the regular triangulation of the packing; every interior throat's entry
    pressure comes from the batched throat LBM (and, as the cheap baseline, from
    incircle and Mayer-Stowe-Princen estimates with sigma from Laplace's law and
    the contact angle of the adhesion estimate); the levels are the reservoir
    capillary pressures the full LBM reached at each of its increments."""
    import torch
    import paper_1906_04722_gb300 as lbm
    import workloads as W

    spheres, box = sample_geometry(args.size)
    params = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                             rho_minor=W.RHO_MINOR, reservoirs=True, membrane_layers=3)
    t_all = time.perf_counter()
    ladder = [W.RHO_MAJOR + 0.02 * i for i in range(20)]
    probe = (box[0] // 2, box[1] // 2, box[2] - 6)
    steps_list = [int(x) for x in str(args.pn_steps).split(",")]
    fulls = {}
    for ns in steps_list:
        dom = lbm.Domain(params, spheres, box)
        mask = dom.mask()
        dom.autotune(trial_steps=10)
        t0 = time.perf_counter()
        fulls[ns] = dom.drainage(ladder, ns, W.RHO_MAJOR, probe)
        torch.cuda.synchronize()
        fulls[ns]["seconds"] = time.perf_counter() - t0
        dom.close()
    full = fulls[steps_list[-1]]
    t_full = sum(f["seconds"] for f in fulls.values())

    t0 = time.perf_counter()
    tets = lbm.lbm_regular_triangulation(spheres)
    vol, tp, ts = lbm.lbm_pn_build(spheres, tets, mask)
    inner = tp[:, 1] >= 0
    tri = spheres[ts[inner]]
    t_net = time.perf_counter() - t0

    tparams = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                              rho_minor=W.RHO_MINOR)
    tl = [W.RHO_MAJOR + 0.02 * i for i in range(32)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.refine > 1:
        _, _, pce_lbm = lbm.lbm_run_throat_batch_refined(tri, tparams, tl, args.throat_steps, W.RHO_MAJOR, args.refine)
    else:
        res, _ = lbm.lbm_run_throat_batch(tri, tparams, tl, args.throat_steps, W.RHO_MAJOR)
        pce_lbm = np.array([r["p_ce"] for r in res])
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    sigma, drops = laplace_sigma(lbm, W)
    from paper_1906_04722_gb300 import surrogate as S
    cos_t = math.cos(S.contact_angle_estimate(W.G_ADS[0], W.G_ADS[1], W.G_COHESION, W.RHO_MAJOR, W.RHO_MINOR))
    pce_inc = lbm.lbm_throat_pce_incircle(tri, sigma, cos_t)
    pce_msp = lbm.lbm_throat_pce_msp(tri, sigma, cos_t)

    levels = np.array([r["p_c_res"] for r in full["rows"]])
    sw_full = np.array([r["S_w"] for r in full["rows"]])

    def network_curve(pce_inner):
        pce = np.zeros(len(tp))
        pce[inner] = pce_inner
        pce[tp[:, 1] == lbm.PN_OUTLET] = np.inf
        sw, inv, trap = lbm.lbm_pn_drainage(vol, tp, pce, levels)
        return sw, int((trap >= 0).sum())

    sw_lbm, trapped_lbm = network_curve(pce_lbm)
    sw_inc, trapped_inc = network_curve(pce_inc)
    sw_msp, trapped_msp = network_curve(pce_msp)
    rows = [{"increment": i, "rho_in_nw": ladder[i], "p_c_res": float(levels[i]), "S_w_full_lbm": float(sw_full[i]),
             "S_w_network_lbm_pce": float(sw_lbm[i]), "S_w_network_incircle": float(sw_inc[i]),
             "S_w_network_msp": float(sw_msp[i])}
            for i in range(len(levels))]
    if len(steps_list) > 1:
        for i, r in enumerate(rows):
            r["S_w_full_lbm_by_steps"] = {str(ns): float(fulls[ns]["rows"][i]["S_w"]) for ns in steps_list}
    fin = np.isfinite(pce_lbm)
    print(json.dumps({
        "workload": f"sample{args.size}: full LBM drainage 20 x {steps_list[-1]} steps vs pore-network drainage "
                    f"on its regular triangulation ({len(tets)} pores, {int(inner.sum())} interior throats); "
                    f"throat ladders 32 x {args.throat_steps} steps"
                    + (f", p_c^e refined to 1/{args.refine} of a ladder step" if args.refine > 1 else ""),
        "seconds": {"full_lbm": t_full, "network_build": t_net, "throat_batch": t_batch,
                    "total": time.perf_counter() - t_all},
        "throats": {"n": int(inner.sum()), "invaded_in_ladder": int(np.isfinite(pce_lbm).sum()),
                    "p_ce_median": float(np.median(pce_lbm[np.isfinite(pce_lbm)])),
                    "incircle_p_ce_median": float(np.median(pce_inc[np.isfinite(pce_inc)])),
                    "incircle_vs_lbm_median_ratio": float(np.median((pce_inc / pce_lbm)[fin])),
                    "msp_p_ce_median": float(np.median(pce_msp[np.isfinite(pce_msp)])),
                    "msp_vs_lbm_median_ratio": float(np.median((pce_msp / pce_lbm)[fin]))},
        "sigma": sigma, "laplace_drops": drops, "cos_theta": cos_t,
        "trapped_pores": {"lbm_pce": trapped_lbm, "incircle": trapped_inc, "msp": trapped_msp},
        "S_w_abs_error": {"lbm_pce_max": float(np.abs(sw_lbm - sw_full).max()),
                          "lbm_pce_mean": float(np.abs(sw_lbm - sw_full).mean()),
                          "incircle_max": float(np.abs(sw_inc - sw_full).max()),
                          "incircle_mean": float(np.abs(sw_inc - sw_full).mean()),
                          "msp_max": float(np.abs(sw_msp - sw_full).max()),
                          "msp_mean": float(np.abs(sw_msp - sw_full).mean())},
        "rows": rows}))
    return 0


def run_surrogate_config5(args):
    """Configuration 5 at its stated size: the throat surrogate trained on 20 k
    throats the batched LBM ran (facets of the regular triangulations of seeded
    300-sphere packings), then asked for 1e5 throats of four seeded 2000-sphere
    packings, the batched LBM taking the throats whose ensemble spread exceeds
    2 %.  The LBM judges a seeded random subset of the 1e5 throats (--judge,
    2000 by default: all of them would take about 5 min of GPU time at 100
    steps per increment); the fallback's cost for all 1e5 is its measured rate
    on that subset's fallback throats.  --train-throats, --throat-steps and
    --refine set the training size, the schedule and the label resolution."""
    import torch
    import paper_1906_04722_gb300 as lbm
    from paper_1906_04722_gb300 import surrogate as S
    import workloads as W

    params = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                             rho_minor=W.RHO_MINOR)
    theta = S.contact_angle_estimate(W.G_ADS[0], W.G_ADS[1], W.G_COHESION, W.RHO_MAJOR, W.RHO_MINOR)
    ladder = [W.RHO_MAJOR + 0.02 * i for i in range(32)]
    n_steps = args.throat_steps
    refine = max(1, args.refine)

    def lbm_pce(th):
        """(results, rows) of the batch; p_ce refined when asked."""
        if refine == 1:
            return lbm.lbm_run_throat_batch(th, params, ladder, n_steps, W.RHO_MAJOR)
        res, rows, fine = lbm.lbm_run_throat_batch_refined(th, params, ladder, n_steps, W.RHO_MAJOR, refine)
        for r, f in zip(res, fine):
            r["p_ce"] = float(f)
        return res, rows

    out = {"workload": "configuration 5: %d training throats of seeded 300-sphere 192^3 packings; 1e5 throats of "
                       "four seeded 2000-sphere 361^3 packings, %d judged by the LBM; 32 increments x %d steps%s; "
                       "5 members, 4 x 256, BF16 operands; fallback at 2 %% ensemble spread"
                       % (args.train_throats, args.judge, n_steps,
                          "" if refine == 1 else ", p_c^e refined to 1/%d of a ladder step" % refine)}
    t0 = time.perf_counter()
    tris, ress, rowss, seed = [], [], [], 110
    while sum(len(t) for t in tris) < args.train_throats:
        th = lbm.packing_throat_sample(W.sample_spheres(192, seed=seed), None, seed)
        res, rows = lbm_pce(th)
        tris.append(th)
        ress += res
        rowss += rows
        seed += 1
    out["training_lbm_s"] = time.perf_counter() - t0
    sur = S.ThroatSurrogate(n_incr=len(ladder), theta=theta, n_members=5, seed=1, spread_tol=0.02)
    t0 = time.perf_counter()
    losses, used = sur.fit(np.concatenate(tris), ress, rowss, epochs=300, batch=256, lr=1e-3, seed=2)
    out["training"] = {"throats": int(sum(len(t) for t in tris)), "used": int(used), "packings": len(tris),
                       "train_s": time.perf_counter() - t0,
                       "loss_first_last": [float(losses[:, 0].mean()), float(losses[:, -1].mean())]}
    inf = np.concatenate([lbm.packing_throat_sample(W.sample_spheres(361, seed=s), None, s) for s in (20, 21, 22, 23)])
    inf = inf[:100000]
    n = len(inf)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pce, rel, _ = sur.predict(inf)
    torch.cuda.synchronize()
    t_net = time.perf_counter() - t0
    fall = rel > 0.02
    sub = np.sort(np.random.default_rng(7).choice(n, min(args.judge, n), replace=False))
    t0 = time.perf_counter()
    truth_res, _ = lbm_pce(inf[sub])
    t_judge = time.perf_counter() - t0
    truth = np.array([r["p_ce"] for r in truth_res])
    fb = sub[fall[sub]]
    t0 = time.perf_counter()
    if len(fb):
        lbm_pce(inf[fb])
    t_fb_sub = time.perf_counter() - t0
    rate_fb = len(fb) / t_fb_sub if len(fb) else float("inf")
    t_fb_all = float(fall.sum()) / rate_fb if len(fb) else 0.0
    answer = np.where(fall[sub], truth, pce[sub])  # fallback throats take the LBM's value
    ok = np.isfinite(truth)
    err_all = np.abs(answer[ok] - truth[ok]) / np.abs(truth[ok])
    ans_ok = ok & ~fall[sub]
    err_ans = np.abs(pce[sub][ans_ok] - truth[ans_ok]) / np.abs(truth[ans_ok])
    plain_th = inf[sub[::max(1, len(sub) // 32)]]
    t0 = time.perf_counter()
    for th in plain_th:
        mask, probe = lbm.lbm_throat_geometry(th)
        d = lbm.Domain(params, mask=mask)
        d.drainage(ladder, n_steps, W.RHO_MAJOR, probe)
        d.close()
    plain = len(plain_th) / (time.perf_counter() - t0)
    value = n / (t_net + t_fb_all)
    out.update({"inference_throats": n, "network_s_all": t_net, "fallback_fraction": float(fall.mean()),
                "fallback_s_all_estimated": t_fb_all, "fallback_rate_throats_per_s": rate_fb,
                "throats_per_s": value, "plain_throats_per_s": plain, "vs_plain": value / plain,
                "batched_lbm_throats_per_s": len(sub) / t_judge,
                "judged_subset": int(len(sub)), "judged_invaded": int(ok.sum()),
                "pce_rel_err_all_median": float(np.median(err_all)), "pce_rel_err_all_p90": float(np.percentile(err_all, 90)),
                "pce_rel_err_answered_median": float(np.median(err_ans)) if err_ans.size else None,
                "pce_rel_err_answered_p90": float(np.percentile(err_ans, 90)) if err_ans.size else None,
                "answered_in_subset": int(ans_ok.sum())})
    # the same predictions under other spread rules (the LBM's answers reused; the
    # fallback's cost scales with the throats it takes at its measured rate)
    sweep = {}
    for tol in (0.02, 0.03, 0.05, 0.1):
        fb_t = rel > tol
        ans_t = ok & ~fb_t[sub]
        e = np.abs(pce[sub][ans_t] - truth[ans_t]) / np.abs(truth[ans_t])
        allv = np.where(fb_t[sub], truth, pce[sub])[ok]
        e_all = np.abs(allv - truth[ok]) / np.abs(truth[ok])
        rate = n / (t_net + float(fb_t.sum()) / rate_fb) if len(fb) else float("nan")
        sweep[f"{tol:g}"] = {"fallback_fraction": float(fb_t.mean()), "throats_per_s": rate,
                             "vs_plain": rate / plain,
                             "answered_median": float(np.median(e)) if e.size else None,
                             "all_median": float(np.median(e_all)), "all_p90": float(np.percentile(e_all, 90))}
    out["spread_rules"] = sweep
    sur.close()
    print(json.dumps(out))
    return 0


def run_throat_convergence(args):
    """Steps per increment for a quasi-static throat ladder (Sec. 2.2.2: the
    density is raised gradually): 64 throats of the held-out packing run the
    32-increment ladder at 100 .. 4000 steps per increment; each p_c^e and
    invasion increment against the 4000-step run."""
    import paper_1906_04722_gb300 as lbm
    import workloads as W

    params = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                             rho_minor=W.RHO_MINOR)
    ladder = [W.RHO_MAJOR + 0.02 * i for i in range(32)]
    tri = lbm.packing_throat_sample(W.sample_spheres(192, seed=3), 64, seed=5)
    runs = {}
    for n_steps in (100, 250, 500, 1000, 2000, 4000):
        t0 = time.perf_counter()
        res, _ = lbm.lbm_run_throat_batch(tri, params, ladder, n_steps, W.RHO_MAJOR)
        runs[n_steps] = ([r["p_ce"] for r in res], [r["invaded_at"] for r in res], time.perf_counter() - t0)
    ref_p, ref_i, _ = runs[4000]
    out = {"workload": "64 throats (regular triangulation) of a 300-sphere 192^3 packing, 32 increments of +0.02",
           "reference": "4000 steps per increment", "rows": []}
    for n_steps, (p, inv, dt) in runs.items():
        both = [k for k in range(len(tri)) if math.isfinite(p[k]) and math.isfinite(ref_p[k])]
        err = [abs(p[k] - ref_p[k]) / abs(ref_p[k]) for k in both]
        out["rows"].append({"steps_per_increment": n_steps, "seconds": dt, "invaded": int(sum(math.isfinite(v) for v in p)),
                            "same_increment_as_ref": int(sum(inv[k] == ref_i[k] for k in range(len(tri)))),
                            "mean_increment_shift": float(np.mean([inv[k] - ref_i[k] for k in both])) if both else None,
                            "pce_rel_diff_median": float(np.median(err)) if err else None,
                            "pce_rel_diff_p90": float(np.percentile(err, 90)) if err else None})
    print(json.dumps(out))
    return 0


def run_throat_batch(args):
    """One lbm_run_throat_batch of the throat benchmark's held-out packing in one
    form, then the same call with zero steps per increment (geometry, lists,
    arenas and the measurements only)."""
    import torch
    import paper_1906_04722_gb300 as lbm
    import workloads as W

    name, *shape = args.throat_batch.split(":")
    form = {"cells": lbm.BATCH_CELLS, "tiles": lbm.BATCH_PER_STEP, "persistent": lbm.BATCH_PERSISTENT,
            "march": lbm.BATCH_MARCH}[name]
    march = (int(shape[0]), int(shape[1])) if shape else (0, 0)  # march:THREADS:PLANES
    params = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                             rho_minor=W.RHO_MINOR)
    ladder = [W.RHO_MAJOR + 0.02 * i for i in range(32)]
    tri = lbm.packing_throat_sample(W.sample_spheres(192, seed=3), None, 3)
    tri = tri[::max(1, len(tri) // max(1, args.throat_count))][:args.throat_count]
    out = {"workload": f"{len(tri)} throats (regular triangulation) of a 300-sphere 192^3 RSA packing, "
                       f"32 increments x {args.throat_steps} steps", "form": args.throat_batch}
    for key, steps in (("full", args.throat_steps), ("no_steps", 0)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, _ = lbm.lbm_run_throat_batch(tri, params, ladder, steps, W.RHO_MAJOR, form=form, march=march)
        torch.cuda.synchronize()
        out[key + "_s"] = time.perf_counter() - t0
    out["throats_per_s"] = len(tri) / out["full_s"]
    out["fluid_cells"] = int(sum(r["n_fluid"] for r in res))
    out["fluid_updates_per_s"] = out["fluid_cells"] * 32 * args.throat_steps / (out["full_s"] - out["no_steps_s"])
    print(json.dumps(out))
    return 0


def main():
    args = parse()
    if args.drainage:
        return run_drainage(args)
    if args.pore_network:
        return run_pore_network(args)
    if args.surrogate_config5:
        return run_surrogate_config5(args)
    if args.throat_convergence:
        return run_throat_convergence(args)
    if args.throat_batch:
        return run_throat_batch(args)
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
