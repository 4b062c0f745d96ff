#!/usr/bin/env python
"""Benchmark: batched encrypted LeNet-1-shaped inference on one GB300.

Workload (the batched LeNet-1 configuration): 633 synthetic 28x28 U[0,1]
images packed 10 per ciphertext (stride 784 slots) into 64 ciphertexts, the
last carrying 3; CKKS N = 16384, chain [60, 40 x 7 | 60], Delta = 2^40,
dnum = 8; LeNet-1 shape conv 1->4 K5, x^2, avgpool 2, conv 4->12 K5, x^2,
avgpool 2, flatten, FC 192->10 with N(0, 0.1^2) weights.

One step = the whole path for the batch: flatten + encode + encrypt of every
sample, the encrypted network (one CUDA graph over all 64 ciphertexts), and
decrypt + decode of the logits.
  value : inputs resident on the device, logits left on the device.
  e2e   : the same through the C ABI with host buffers (pinned input copied in,
          logits copied out inside the timed region).
  plain : the one-op-per-launch path (each ciphertext through the layers on
          its own, eager launches, no graph), per-sample rate on a sample.
Timing: CUDA events on the library's stream after warm-up; every step's
working set (keys ~1.7 GB, cached plaintext masks ~1.3 GB, ciphertexts) is far
larger than the 126 MB L2.

--impl reference runs the CPU oracle (oracle/, plain C with __int128 '%') on a
bounded sample of the same workload on this host's cores: K steps of one
ciphertext each, on min(K, cores) concurrent single-threaded processes.
--ncu-step / --ncu-conv run one eager step / one conv2d layer call between
cudaProfilerStart and cudaProfilerStop for `ncu --profile-from-start off`.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

N_SAMPLES = 633
TUNE_CACHE = os.path.join(ROOT, "paper_2402_03060_gb300", "_build", "tune_cache.json")
# DRAM traffic of the dominant kernels as a ratio to their algorithmic bytes, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum, few metrics, one kernel family and at most 16
# launches) on the small `--ncu-conv` case; the line's per-launch traffic is that ratio times the
# kernel's algorithmic bytes per launch in the benchmark step (the traffic of these kernels grows
# in proportion to the rows they convert and transform).  Valid only for the kernel sources (the
# hashed functions) and limb layout it was taken with, else reported as null.
NCU_TRAFFIC = {
    "modup_ntt": {
        # one ModUp of 4 x 8 ciphertexts at N = 2^14, lp = 8, dnum = 8: 2048 converted rows;
        # modup2_outer_kernel<4> 33.7 MB read + 207.8 MB written, its ntt2_inner_kernel 271.1 MB
        # read + 207.6 MB written = 720.2 MB against 8 N rows (1 + alpha) = 536.9 MB algorithmic
        "dram_per_algorithmic_byte": 720.2 / 536.9,
        "sources": [("paper_2402_03060_gb300/csrc/keyswitch.cu",
                     "template <int R>\n__global__ void __launch_bounds__(NTT2_COLS) modup2_outer_kernel("),
                    ("paper_2402_03060_gb300/csrc/ntt.cu",
                     "__global__ void __launch_bounds__(NTT2_INNER_THREADS) ntt2_inner_kernel(")],
        "tuning": {"ntt_split": 2},
    },
}
# SHA-256 of each source function above as measured
NCU_TRAFFIC_SHA = {"modup_ntt": ["2bc7722999b319be04e41f98b7b3cfec2abcdc1ecc770a71d6d2d873e9fcc0e5",
                                 "0fbcef6e7900a8c07ea3418d05a135eae1112eef0d2acd3acaada72cdf26a5e6"]}


def kernel_hash(path, start):
    """SHA-256 of one kernel's source text: from `start` to the brace closing its body."""
    import hashlib
    with open(os.path.join(ROOT, path)) as f:
        src = f.read()
    i = src.find(start)
    if i < 0:
        return None
    j = src.index("{", src.index(")", i))
    depth = 0
    for k in range(j, len(src)):
        depth += {"{": 1, "}": -1}.get(src[k], 0)
        if depth == 0:
            return hashlib.sha256(src[i:k + 1].encode()).hexdigest()
    return None


def ncu_traffic(kernel, tuning, alg_bytes_per_launch):
    """Per-launch DRAM traffic of kernel: the stored ratio times its algorithmic bytes per launch,
    if the kernel sources and limb layout are the ones it was measured with, else None."""
    t = NCU_TRAFFIC.get(kernel)
    if not t:
        return None
    hashes = [kernel_hash(path, fn) for path, fn in t["sources"]]
    if hashes != NCU_TRAFFIC_SHA.get(kernel):
        return None
    if any(tuning.get(k) != v for k, v in t["tuning"].items()):
        return None
    return round(t["dram_per_algorithmic_byte"] * alg_bytes_per_launch)


SPC = 10
METRIC = "encrypted LeNet-1 inferences/s (batched)"
UNIT = "samples/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the one-op-per-launch comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--samples", type=int, default=N_SAMPLES)
    ap.add_argument("--keys", default="step", choices=["step", "pow2"],
                    help="Galois keys: one per rotation step (default) or the power-of-two set")
    ap.add_argument("--schedule", default="fused", choices=["fused", "literal"],
                    help="evaluation schedule: fused (default) or the paper's order, one operation at a time")
    ap.add_argument("--ncu-step", action="store_true",
                    help="after set-up and warm-up run ONE eager step between cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off) and exit")
    ap.add_argument("--serve", action="store_true",
                    help="serving benchmark instead: Poisson arrivals over a LeNet-1 / LeNet-5 / 1-D CNN mix through "
                         "the continuous-batching loop; prints request-latency percentiles")
    ap.add_argument("--requests", type=int, default=600, help="requests of the --serve trace")
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests of the default run's short serving trace")
    ap.add_argument("--no-serve", action="store_true", help="skip the default run's serving leg")
    ap.add_argument("--rate", type=float, default=200.0, help="arrivals per second of the --serve trace")
    ap.add_argument("--serve-max-batch", type=int, default=8, help="ciphertexts per batch of one model")
    ap.add_argument("--serve-inflight", type=int, default=1, help="batches of one model in flight")
    ap.add_argument("--serve-padded", action="store_true",
                    help="pad batches to a power of two (default: one graph per exact batch size)")
    ap.add_argument("--ncu-conv", action="store_true",
                    help="small case for full ncu captures: ONE hoisted conv2d layer call (4 -> 12 channels, 5x5, "
                         "8 ciphertexts per channel, N = 16384, top level) between cudaProfilerStart/Stop, then exit")
    ap.add_argument("--ncu-cts", type=int, default=8, help="ciphertexts per channel of the --ncu-conv case")
    ap.add_argument("--mac-tc", type=int, default=-1,
                    help="--ncu-conv: the mac_tc tuning knob (0 integer MAC, 5 the 40-bit limbs on the tensor cores, "
                         "8 every limb); default: the library's")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def lenet_setup(G, torch, device, stream, n_samples, keys="step", schedule="fused"):
    P = W.PARAMS["lenet1"]
    model = W.lenet1()
    stride, levels, steps = G.plan(model, 28, 28, schedule=schedule)
    ctx = G.Context(seed=W.KEY_SEED, device=device, stream=stream.cuda_stream, **P)
    ctx.autotune(TUNE_CACHE)
    ctx.set_schedule(schedule)
    if keys == "pow2":
        ctx.keygen_pow2()   # the power-of-two key set: rotations as non-adjacent-form chains
    else:
        ctx.keygen(steps)
    m = ctx.compile(model, 28, 28, SPC)
    imgs = W.images(n_samples)
    return ctx, m, stride, model, imgs


def conv_case(args, local):
    """The second LeNet-1 convolution's shape as one layer call: 25 rotation keys,
    4 input channels x 8 ciphertexts (--ncu-cts), 12 output channels (about 2.5 GB on the device),
    followed by a 2x2 average pooling of the same 4 x 8 ciphertexts (the one-pass
    combination of three rotations and the identity)."""
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_03060_gb300 as G
    P = W.PARAMS["lenet1"]
    w = W.lenet1()[3]
    stream = torch.cuda.Stream()
    ctx = G.Context(seed=W.KEY_SEED, device=local, stream=stream.cuda_stream, **P)
    ctx.keygen(sorted({k + 28 * j for j in range(5) for k in range(5)} - {0}))
    if args.mac_tc >= 0:
        ctx.set_tuning(mac_tc=args.mac_tc)
    imgs = W.images(SPC * args.ncu_cts)
    cts = [ctx.encrypt(imgs, SPC, 784, W.ENC_SEED + c) for c in range(4)]
    for _ in range(max(args.warmup, 1)):
        ctx.conv2d(cts, w["w"], w["b"])
        ctx.avgpool(cts, 2)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    ctx.conv2d(cts, w["w"], w["b"])
    ctx.avgpool(cts, 2)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    return {"ncu_conv": True}


SERVE_MODELS = (  # name, layers, image W, H, samples per ciphertext, logits
    ("lenet1", W.lenet1, 28, 28, 10, 10),
    ("lenet5", W.lenet5_sq, 32, 32, 16, 10),
    ("cnn1d", lambda: W.cnn1d(fc_sum="tree"), 1024, 1, 2, 5),
)


def run_serve(args, local, requests=None, full=True):
    """Poisson(rate) requests, each one sample of a uniformly drawn model; the
    clients' ciphertexts are encrypted beforehand and submitted to the serving
    loop at their arrival times; a second thread collects the results.
    Latency = submit to completion on the device.  full=False (the default
    benchmark's serving leg): the main trace only, no per-layer breakdown and no
    second trace at 80 % of capacity."""
    requests = requests or args.requests
    import threading
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_03060_gb300 as G
    t_setup = time.perf_counter()
    srv = G.Server(max_batch=args.serve_max_batch, max_wait_us=2000, max_inflight=args.serve_inflight,
                   exact_batches=not args.serve_padded)
    ctxs, models, strides, layers = [], [], [], []
    for i, (name, fn, Wi, Hi, spc, nout) in enumerate(SERVE_MODELS):
        ly = fn()
        stride, levels, steps = G.plan(ly, Wi, Hi)
        ctx = G.Context(seed=W.KEY_SEED, device=local, **W.SERVE_PARAMS[name])
        ctx.autotune(TUNE_CACHE)
        ctx.keygen(steps)
        m = ctx.compile(ly, Wi, Hi, spc)
        assert srv.add_model(m) == i
        ctxs.append(ctx)
        models.append(m)
        strides.append(stride)
        layers.append(ly)
    t_setup = time.perf_counter() - t_setup
    # service cost of each model: one graph-launched batch of 1 and of 8 ciphertexts, and the
    # per-layer split of one eager batch of 8 (CUDA events per launch)
    service = {}
    for i, (name, fn, Wi, Hi, spc, nout) in enumerate(SERVE_MODELS):
        ctx = ctxs[i]
        x = W.images(8 * spc, Hi, Wi) if Hi > 1 else W.signals(8 * spc, Wi)
        row = {}
        for b in (1, 8):
            ct = ctx.encrypt(x[:b * spc], spc, strides[i], W.ENC_SEED)
            models[i].infer(ct, use_graph=True)
            ctx.sync()
            t = time.perf_counter()
            for _ in range(3):
                models[i].infer(ct, use_graph=True)
            ctx.sync()
            row[f"ms_batch{b}"] = round((time.perf_counter() - t) / 3 * 1e3, 2)
        ct = ctx.encrypt(x, spc, strides[i], W.ENC_SEED)
        tagged = {}
        if full:
            ctx.profile_begin()
            models[i].infer(ct)
            tagged = ctx.profile_end()
        layers_ms, kern_ms = {}, {}
        for key, (nl, ms, byt, ops) in tagged.items():
            lay, _, kern = key.rpartition("/")
            layers_ms[lay or "other"] = round(layers_ms.get(lay or "other", 0.0) + ms, 2)
            kern_ms[kern] = round(kern_ms.get(kern, 0.0) + ms, 2)
        if full:
            row["eager_batch8_layers_ms"] = layers_ms
            row["eager_batch8_kernels_ms"] = dict(sorted(kern_ms.items(), key=lambda kv: -kv[1])[:8])
        service[name] = row
    def trace(rate, n, seed):
        """Replay n Poisson(rate) arrivals; latencies as the loop reports them."""
        rng = np.random.default_rng(seed)
        arrival = np.cumsum(rng.exponential(1.0 / rate, n))
        which = rng.integers(0, len(SERVE_MODELS), n)
        # the clients' ciphertexts: encrypted before the trace starts (client-side work)
        cts = []
        for k in range(n):
            i = which[k]
            name, fn, Wi, Hi, spc, nout = SERVE_MODELS[i]
            x = W.images(1, Hi, Wi, seed=W.INPUT_SEED + k) if Hi > 1 else W.signals(1, Wi, seed=W.INPUT_SEED + k)
            cts.append(ctxs[i].encrypt(x, spc, strides[i], W.ENC_SEED + k))
        for c in ctxs:
            c.sync()
        ids = [None] * n
        lat = np.zeros(n)
        done_t = np.zeros(n)
        results = {}
        ready = threading.Semaphore(0)

        def collect():
            for k in range(n):
                ready.acquire()
                out, lat[k] = srv.wait(ids[k], 600000)
                done_t[k] = time.perf_counter()
                if which[k] not in results:
                    results[which[k]] = (k, out)
        th = threading.Thread(target=collect)
        th.start()
        t0 = time.perf_counter()
        for k in range(n):
            delay = t0 + arrival[k] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids[k] = srv.submit(int(which[k]), cts[k])
            cts[k] = None
            ready.release()
        th.join()

        def pct(v, p):   # nearest rank
            v = np.sort(v)
            return float(v[max(0, int(np.ceil(p * len(v))) - 1)]) if len(v) else 0.0
        per_model = {}
        for i, (name, *_rest) in enumerate(SERVE_MODELS):
            li = lat[which == i]
            per_model[name] = {"requests": int(len(li)), "p50_ms": round(pct(li, 0.5), 2),
                               "p99_ms": round(pct(li, 0.99), 2), "max_ms": round(float(li.max()), 2) if len(li) else 0}
        # first result of each model decrypted (correctness of what was served)
        for i, (k, out) in results.items():
            nout = SERVE_MODELS[i][5]
            per_model[SERVE_MODELS[i][0]]["first_result_logits"] = [round(float(v), 4) for v in
                                                                    ctxs[i].decrypt(out, nout)[0][:3]]
        return {"rate_per_s": rate, "requests": n, "p50_ms": round(pct(lat, 0.5), 3),
                "p99_ms": round(pct(lat, 0.99), 3), "max_ms": round(float(lat.max()), 3),
                "throughput_req_per_s": round(n / (done_t.max() - t0), 2), "per_model": per_model}

    offered = args.rate / len(SERVE_MODELS) * sum(v["ms_batch8"] / 8 for v in service.values()) / 1e3
    main = trace(args.rate, requests, W.ARRIVAL_SEED)
    st = srv.stats()
    for i, (name, *_rest) in enumerate(SERVE_MODELS):
        si = srv.stats(i)
        main["per_model"][name].update({"batches": si["batches"], "mean_batch_cts": round(si["mean_batch"], 2)})
    knee = None
    if full:
        # the same mix at 80 % of the capacity the batch-of-8 service costs allow
        knee_rate = round(0.8 * args.rate / max(offered, 1e-9), 1)
        knee = trace(knee_rate, requests, W.ARRIVAL_SEED + 1)
    srv.close()
    return {"metric": "serving request latency p99 (Poisson arrivals, LeNet-1 / LeNet-5 / 1-D CNN mix)",
            "value": main["p99_ms"], "unit": "ms", "n_gpus": 1, "higher_is_better": False,
            "p50_ms": main["p50_ms"], "max_ms": main["max_ms"], "throughput_req_per_s": main["throughput_req_per_s"],
            "requests": requests, "rate_per_s": args.rate,
            "loop_stats": {"p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                           "mean_batch_cts": round(st["mean_batch"], 2), "batches": st["batches"]},
            "dtype": "u64 (RNS residues), f64 encode", "data": "synthetic",
            "config": {"workload": "serving mix, one sample per request",
                       "models": {m[0]: W.SERVE_PARAMS[m[0]] for m in SERVE_MODELS},
                       "max_batch_cts": args.serve_max_batch, "max_wait_us": 2000,
                       "max_inflight_per_model": args.serve_inflight,
                       "batches": "padded to a power of two" if args.serve_padded else "exact sizes",
                       "arrival_seed": W.ARRIVAL_SEED},
            "setup_s": round(t_setup, 1), "per_model": main["per_model"], "service_cost": service,
            "offered_load": round(offered, 3), "at_80pct_capacity": knee}


def max_over_ranks(vals, dist, device):
    """Element-wise maximum of the per-rank timings (every rank gets it); replicas
    exchange nothing else."""
    if dist is None:
        return list(vals)
    import torch
    t = torch.tensor(list(vals), device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def whole_job_rate(samples_per_rank, world, ms_step_max):
    """Weak scaling: every rank processes its own batch; the job's rate is all
    ranks' samples over the slowest rank's step time."""
    return samples_per_rank * world / (ms_step_max / 1e3)


def run_ours(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_03060_gb300 as G

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    stream = torch.cuda.Stream()
    ctx, model, stride, layers, imgs = lenet_setup(G, torch, local, stream, args.samples, args.keys, args.schedule)
    n_ct = -(-args.samples // SPC)
    x_dev = torch.from_numpy(imgs).to(f"cuda:{local}")
    x_host = torch.from_numpy(imgs).pin_memory()
    logits_dev = torch.zeros((n_ct * SPC, 10), dtype=torch.float64, device=f"cuda:{local}")
    seed = W.ENC_SEED + 100000 * rank

    def step_device():
        ct = ctx.encrypt(x_dev, SPC, stride, seed)
        out = model.infer(ct, use_graph=True)
        ctx.decrypt(out, 10, out=logits_dev)
        return out

    def step_e2e():
        ct = ctx.encrypt(x_host.numpy(), SPC, stride, seed)
        out = model.infer(ct, use_graph=True)
        return ctx.decrypt(out, 10)

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(fn, k):
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        barrier()
        return e0.elapsed_time(e1), wall * 1e3

    for _ in range(max(args.warmup, 3)):
        step_device()
    if args.ncu_step:
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        ct = ctx.encrypt(x_dev, SPC, stride, seed)
        out = model.infer(ct, use_graph=False)
        ctx.decrypt(out, 10, out=logits_dev)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        return {"ncu_step": True, "samples": args.samples}, ctx
    # logits of the measured configuration (checked against the FP64 CNN in the CPU-baseline leg)
    torch.cuda.synchronize()
    chk = logits_dev.cpu().numpy()

    clocks = Clocks(local)
    launches0 = ctx.launches()
    clocks.start()
    ms_dev, _ = timed(step_device, args.steps)
    clk = clocks.stop()
    launches = (ctx.launches() - launches0) // max(1, args.steps)

    for _ in range(2):
        step_e2e()
    ms_e2e_ev, ms_e2e_wall = timed(step_e2e, args.steps)

    # per-kernel CUDA-event timing of one eager step (roofline of the dominant kernel)
    ctx.profile_begin()
    ct = ctx.encrypt(x_dev, SPC, stride, seed)
    out = model.infer(ct, use_graph=False)
    ctx.decrypt(out, 10, out=logits_dev)
    tagged = ctx.profile_end()
    # records are "layer/kernel" (or "kernel" outside the network): totals per kernel and per layer
    stats, layer_ms = {}, {}
    for key, (nl, ms, byt, ops) in tagged.items():
        layer, _, kern = key.rpartition("/")
        s = stats.setdefault(kern, [0, 0.0, 0.0, 0.0])
        s[0] += nl
        s[1] += ms
        s[2] += byt
        s[3] += ops
        lk = layer or "encrypt/decrypt"
        layer_ms[lk] = layer_ms.get(lk, 0.0) + ms
    # measured integer roofline: register-only throughput of the primitives
    bfly_peak, mac_peak, _barrett_peak, ub_sms = ctx.ubench()
    stats = {k: tuple(v) for k, v in stats.items()}

    # one-op-per-launch path: each ciphertext alone, eager
    plain = None
    if not args.no_plain:
        k = 4
        cts = [ctx.encrypt(x_dev[SPC * i: SPC * (i + 1)], SPC, stride, seed + i) for i in range(k)]
        model.infer(cts[0])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for c in cts:
            model.infer(c, use_graph=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        plain = {"value": k * SPC / (ms / 1e3), "unit": UNIT, "ms_per_ct": ms / k,
                 "sample": f"{k} ciphertexts x {SPC} samples, one ciphertext per launch, eager"}

    # max over ranks
    ms_step, ms_e2e = max_over_ranks([ms_dev / args.steps, ms_e2e_wall / args.steps], dist, f"cuda:{local}")
    total_samples = args.samples * world
    pk = peaks()
    roof = None
    if stats:
        peak_hbm = pk["hbm_gbs"] if pk else 6800.0
        alu_peak = {"ntt": bfly_peak, "intt": bfly_peak, "moddown": bfly_peak, "rescale": bfly_peak,
                    "modup_ntt": bfly_peak,
                    "mac": mac_peak, "ks_lazy": mac_peak, "ks_inner": mac_peak, "ks_comb": mac_peak}

        def views(v):
            nl, tms, byt, ops = v
            if tms <= 0:
                return None, None
            gbs = byt / (tms / 1e3) / 1e9
            return gbs, (ops / (tms / 1e3))

        kern_rows = {}
        for k, v in sorted(stats.items(), key=lambda kv: -kv[1][1]):
            gbs, opss = views(v)
            row = {"launches": v[0], "ms": round(v[1], 3), "GBps": round(gbs, 1) if gbs else None,
                   "hbm_frac": round(gbs / peak_hbm, 4) if gbs else None}
            if k in alu_peak and opss:
                row["ops_per_s"] = float(f"{opss:.4g}")
                row["alu_frac"] = round(opss / alu_peak[k], 4)
            kern_rows[k] = row
        name, v = max(stats.items(), key=lambda kv: kv[1][1])
        nl, tms, byt, ops = v
        share = tms / sum(x[1] for x in stats.values())
        gbs, opss = views(v)
        hbm_frac = gbs / peak_hbm
        alu_frac = opss / alu_peak[name] if name in alu_peak and opss else 0.0
        if alu_frac > hbm_frac:
            unit = "Gbutterfly/s" if alu_peak[name] is bfly_peak else "G(64x64->128 MAC)/s"
            roof = {"bound": "alu", "kernel": name, "achieved": round(opss / 1e9, 2),
                    "peak": round(alu_peak[name] / 1e9, 2), "unit": unit, "frac": round(alu_frac, 4),
                    "peak_source": "measured register-only primitive throughput (he_ubench) on this GPU",
                    "hbm_view": {"achieved_GBps": round(gbs, 1), "peak_GBps": peak_hbm, "frac": round(hbm_frac, 4),
                                 "peak_source": "measured (MEASURED_PEAKS.json)" if pk else
                                 "fallback 6800 GB/s (MEASURED_PEAKS.json absent)"}}
        else:
            roof = {"bound": "hbm", "kernel": name, "achieved": round(gbs, 1), "peak": peak_hbm, "unit": "GB/s",
                    "frac": round(hbm_frac, 4), "peak_source": "measured" if pk else "fallback"}
        roof.update({"traffic": ncu_traffic(name, ctx.tuning(), byt / nl), "launches_per_step": nl, "avg_launch_us": round(tms / nl * 1e3, 2),
                     "share_of_eager_step": round(share, 3),
                     "primitive_peaks": {"butterflies_per_s": float(f"{bfly_peak:.4g}"),
                                         "mac128_per_s": float(f"{mac_peak:.4g}"),
                                         "barrett_per_s": float(f"{_barrett_peak:.4g}"), "sm_count": int(ub_sms)}})
    profile = {"kernels": kern_rows if stats else {},
               "layers_ms": {k: round(v, 3) for k, v in layer_ms.items()},
               "top_layer_kernels_ms": {k: round(v[1], 3) for k, v in
                                        sorted(tagged.items(), key=lambda kv: -kv[1][1])[:12]}}
    res = {
        "metric": METRIC, "value": round(whole_job_rate(args.samples, world, ms_step), 3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64 (RNS residues), f64 encode",
        "data": "synthetic U[0,1] 28x28 images, N(0,0.1^2) weights (MNIST / trained weights absent)",
        "config": {"workload": "batched LeNet-1-shaped, 64 ciphertexts x 10 samples (last 3), 633 samples",
                   "ckks": "N=16384, [60,40x7|60], Delta=2^40, dnum=8", "samples_per_gpu": args.samples,
                   "galois_keys": ("power of two (+-2^k), rotations as non-adjacent-form chains"
                                   if args.keys == "pow2" else "one per rotation step of the model"),
                   "schedule": args.schedule,
                   "l2": "working set > L2 (keys + masks + ciphertexts, several GB)",
                   "parallelism": f"replicas x{world}", "autotuned": ctx.tuning()},
        "e2e": {"value": round(total_samples / (ms_e2e / 1e3), 3), "unit": UNIT,
                "h2d_bytes_per_step": int(args.samples * 784 * 8), "d2h_bytes_per_step": int(n_ct * SPC * 10 * 8)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "profile": profile,
        "clocks": clk,
        "plain": round(plain["value"], 3) if plain else None,
        "plain_detail": plain,
    }
    res["_logits"] = (chk, imgs, layers)
    return res, ctx


def oracle_sample():
    """The CPU oracle on one ciphertext (10 samples) of the workload; keys are
    generated first (not timed, like the GPU's).  Returns (samples/s, seconds, note)."""
    he, pl, model = _oracle_setup()
    t = _oracle_step(he, pl, model)
    return SPC / t, t, "one ciphertext (10 samples) end to end: encrypt, LeNet-1, decrypt; keygen untimed"


def _oracle_setup():
    from oracle import ckks, layers
    P = W.PARAMS["lenet1"]
    model = W.lenet1()
    pl = layers.plan(model, 28, 28)
    he = ckks.Ckks(seed=W.KEY_SEED, **P)
    he.keygen(pl["steps"])
    return he, pl, model


def _oracle_step(he, pl, model) -> float:
    """One step of the reference arm: encrypt, run and decrypt one ciphertext of
    10 samples with the oracle; returns its seconds."""
    from oracle import layers
    imgs = W.images(SPC)
    lay = layers.input_layout(28, 28, pl["stride"], SPC, he.n // 2)
    x = np.zeros(he.n // 2)
    for b in range(SPC):
        x[b * pl["stride"]: b * pl["stride"] + 784] = imgs[b].reshape(-1)
    t0 = time.perf_counter()
    ct = he.encrypt(x, W.ENC_SEED)
    ys, _ = layers.run_model(layers.HeBackend(he), ct, model, lay)
    he.decrypt(ys[0])
    return time.perf_counter() - t0


def _oracle_worker(n_steps, barrier, out):
    """Spawned process: keygen (its warm-up, untimed), wait for every worker,
    then n_steps timed oracle steps; reports (start, end) on the monotonic clock."""
    os.environ["OMP_NUM_THREADS"] = "1"
    he, pl, model = _oracle_setup()
    barrier.wait()
    t0 = time.monotonic()
    for _ in range(n_steps):
        _oracle_step(he, pl, model)
    out.put((t0, time.monotonic()))


def run_reference(args):
    """The reference arm: the oracle as it stands, K steps of one ciphertext each,
    spread over min(K, host cores) single-threaded processes that start together."""
    import multiprocessing as mp
    from oracle import build as oracle_build
    oracle_build.build()  # once, before the workers load it
    k = max(1, args.steps)
    procs = max(1, min(k, os.cpu_count() or 1))
    per = [k // procs + (1 if i < k % procs else 0) for i in range(procs)]
    sp = mp.get_context("spawn")
    barrier, q = sp.Barrier(procs), sp.Queue()
    ps = [sp.Process(target=_oracle_worker, args=(n, barrier, q)) for n in per]
    for p in ps:
        p.start()
    spans = [q.get() for _ in ps]
    for p in ps:
        p.join()
    t = max(e for _, e in spans) - min(s for s, _ in spans)
    v = k * SPC / t
    note = (f"{k} steps of one ciphertext (10 samples) each, end to end (encrypt, LeNet-1, decrypt), on "
            f"{procs} concurrent single-threaded processes; each process generates its keys first (untimed, "
            "its warm-up)")
    return {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": UNIT, "n_gpus": 1,
            "steps": k, "warmup": 0, "ms_per_step": round(t * 1e3 / k, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64 (RNS residues), f64 encode",
            "data": "synthetic U[0,1] 28x28 images, N(0,0.1^2) weights",
            "config": {"workload": "batched LeNet-1-shaped, one ciphertext of 10 samples per step",
                       "ckks": "N=16384, [60,40x7|60], Delta=2^40, dnum=8"},
            "cpu_baseline": {"value": round(v, 5), "unit": UNIT, "cores": procs, "kind": "oracle", "sample": note},
            "e2e": {"value": round(v, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if args.ncu_conv:
        print(json.dumps(conv_case(args, local)))
        return
    if args.serve:
        if rank == 0:
            print(json.dumps(run_serve(args, local)))
        return
    res, ctx = run_ours(args, rank, world, local)
    if args.ncu_step:
        print(json.dumps(res))
        return
    chk, imgs, layers = res.pop("_logits", (None, None, None))
    if rank == 0 and world == 1 and not args.no_cpu:
        v, t, note = oracle_sample()
        res["cpu_baseline"] = {"value": round(v, 5), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": note,
                               "seconds": round(t, 1)}
        # the timed configuration's logits against the FP64 CNN on a spread of samples
        from oracle import cnn
        worst = 0.0
        for k in list(range(0, len(imgs), max(1, len(imgs) // 7)))[:8] + [len(imgs) - 1]:
            worst = max(worst, float(np.abs(chk[k] - cnn.forward(imgs[k], layers)).max()))
        res["max_abs_logit_err_vs_fp64"] = worst
    if rank == 0 and world == 1 and not args.no_serve:
        # the serving mix (Poisson arrivals over LeNet-1 / LeNet-5 / 1-D CNN, continuous batching),
        # a short trace: request latency percentiles beside the batched throughput
        del ctx
        try:
            sv = run_serve(args, local, requests=args.serve_requests, full=False)
            res["serve"] = {"p50_ms": sv["p50_ms"], "p99_ms": sv["value"], "max_ms": sv["max_ms"],
                            "throughput_req_per_s": sv["throughput_req_per_s"], "requests": sv["requests"],
                            "rate_per_s": sv["rate_per_s"], "offered_load": sv["offered_load"],
                            "mean_batch_cts": sv["loop_stats"]["mean_batch_cts"], "setup_s": sv["setup_s"],
                            "workload": "Poisson arrivals, one-sample requests, uniform LeNet-1 (N=2^14) / "
                                        "LeNet-5 (N=2^15) / 1-D CNN (N=2^14) mix, dnum=3 keys resident, "
                                        "max 8 ciphertexts per batch"}
        except Exception as e:   # the throughput line stands without it
            res["serve"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    if rank == 0:
        # the bulky per-kernel profile first, the headline extras last (short tails stay readable)
        order = [k for k in res if k not in ("profile", "plain_detail", "cpu_baseline", "max_abs_logit_err_vs_fp64",
                                             "clocks", "plain", "serve")]
        tail = ["profile", "plain_detail", "cpu_baseline", "max_abs_logit_err_vs_fp64", "clocks", "plain", "serve"]
        print(json.dumps({k: res[k] for k in order + [k for k in tail if k in res]}))


if __name__ == "__main__":
    main()
