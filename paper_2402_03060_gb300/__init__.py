"""GB300 (sm_103a) library for UniHENN's encrypted CNN inference (arXiv 2402.03060).

The Python layer only marshals arguments to the C ABI of libunihenn.so
(include/unihenn.h); every step of the RNS-CKKS path runs in its CUDA kernels.
Device memory for ciphertexts and keys is owned by the library's pool;
inputs may be host numpy arrays or CUDA torch tensors.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import _lib
from ._lib import HeError, check, load

__all__ = ["Context", "Ct", "Model", "Server", "HeError", "layers_to_c", "plan", "load", "simulate_server"]


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Ct:
    """A batch of ciphertexts (one he_ct handle)."""

    def __init__(self, ctx: "Context", h):
        self.ctx = ctx
        self.h = ctypes.c_void_p(h) if not isinstance(h, ctypes.c_void_p) else h

    def info(self):
        b, l, s = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_double()
        check(load().he_ct_info(self.h, ctypes.byref(b), ctypes.byref(l), ctypes.byref(s)))
        return b.value, l.value, s.value

    @property
    def batch(self):
        return self.info()[0]

    @property
    def limbs(self):
        return self.info()[1]

    @property
    def scale(self):
        return self.info()[2]

    def free(self):
        if self.h is not None and self.h.value:
            load().he_ct_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def layers_to_c(layers):
    """workloads-style layer dicts -> (he_layer array, kept numpy buffers)."""
    keep = []
    arr = (_lib.he_layer * len(layers))()
    for i, l in enumerate(layers):
        op = l["op"]
        e = arr[i]
        if op in ("conv2d", "conv1d"):
            w = np.ascontiguousarray(l["w"], dtype=np.float64)
            b = np.ascontiguousarray(l["b"], dtype=np.float64)
            keep += [w, b]
            e.op = _lib.HE_CONV2D if op == "conv2d" else _lib.HE_CONV1D
            e.ch_out, e.ch_in, e.k = w.shape[0], w.shape[1], w.shape[-1]
            e.stride = l["stride"]
            e.w, e.b = _dptr(w), _dptr(b)
        elif op == "fc":
            w = np.ascontiguousarray(l["w"], dtype=np.float64)
            b = np.ascontiguousarray(l["b"], dtype=np.float64)
            keep += [w, b]
            e.op = _lib.HE_FC
            e.ch_out, e.ch_in = w.shape
            e.k = {"linear": 0, "tree": 1}[l.get("sum", "linear")]
            e.w, e.b = _dptr(w), _dptr(b)
        elif op == "square":
            e.op = _lib.HE_SQUARE
        elif op == "approx_relu":
            e.op = _lib.HE_APPROX_RELU
        elif op == "avgpool":
            e.op = _lib.HE_AVGPOOL
            e.k = l["k"]
        elif op == "flatten":
            e.op = _lib.HE_FLATTEN
        else:
            raise ValueError(op)
    return arr, keep


def plan(layers, W_img: int, H_img: int, schedule: str = "fused"):
    """he_model_plan_schedule: (stride, levels, rotation steps); schedule "fused" or "literal"."""
    arr, keep = layers_to_c(layers)
    L = load()
    sc = _lib.SCHEDULES[schedule]
    stride, levels, n = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_size_t(0)
    check(L.he_model_plan_schedule(arr, len(layers), W_img, H_img, sc, ctypes.byref(stride), ctypes.byref(levels),
                                   None, ctypes.byref(n)))
    steps = (ctypes.c_int32 * n.value)()
    check(L.he_model_plan_schedule(arr, len(layers), W_img, H_img, sc, None, None, steps, ctypes.byref(n)))
    return stride.value, levels.value, list(steps)


def pack_steps(stride: int, n: int):
    """Rotation steps he_pack needs for n one-sample ciphertexts: right by k*stride."""
    return [-k * stride for k in range(1, n)]


class Model:
    def __init__(self, ctx: "Context", h, keep):
        self.ctx, self._keep = ctx, keep
        self.h = h if isinstance(h, ctypes.c_void_p) else ctypes.c_void_p(h)

    def set_mask_budget(self, nbytes: int):
        """he_model_set_mask_budget: encode a convolution's masks per inference when they
        would take more than nbytes (0: keep every mask)."""
        check(load().he_model_set_mask_budget(self.h, nbytes))

    def infer(self, ct: Ct, use_graph: bool = False) -> Ct:
        out = ctypes.c_void_p()
        check(load().he_infer(self.h, ct.h, int(use_graph), ctypes.byref(out)))
        return Ct(self.ctx, out)

    def free(self):
        if self.h is not None and self.h.value:
            load().he_model_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """he_server_*: continuous-batching request loop over compiled models."""

    def __init__(self, max_batch: int = 8, max_wait_us: int = 0, mem_budget: int = 0, max_inflight: int = 0,
                 exact_batches: bool = False):
        self._models, self._req_ctx = [], {}
        opt = _lib.he_server_opts(max_batch, max_wait_us, mem_budget, max_inflight, int(exact_batches))
        h = ctypes.c_void_p()
        check(load().he_server_create(ctypes.byref(opt), ctypes.byref(h)))
        self.h = h

    def add_model(self, model: Model) -> int:
        mid = ctypes.c_uint32()
        check(load().he_server_add_model(self.h, model.h, ctypes.byref(mid)))
        self._models.append(model)
        return mid.value

    def submit(self, model_id: int, ct: Ct) -> int:
        rid = ctypes.c_uint64()
        check(load().he_server_submit(self.h, model_id, ct.h, ctypes.byref(rid)))
        self._req_ctx[rid.value] = self._models[model_id].ctx
        return rid.value

    def poll(self, req_id: int) -> bool:
        done = ctypes.c_int()
        check(load().he_server_poll(self.h, req_id, ctypes.byref(done)))
        return bool(done.value)

    def wait(self, req_id: int, timeout_ms: int = 60000):
        """-> (result Ct, latency in ms)"""
        out, lat = ctypes.c_void_p(), ctypes.c_double()
        check(load().he_server_wait(self.h, req_id, timeout_ms, ctypes.byref(out), ctypes.byref(lat)))
        return Ct(self._req_ctx.pop(req_id), out), lat.value

    def stats(self, model_id: int = -1) -> dict:
        st = _lib.he_server_stats()
        check(load().he_server_stats_get(self.h, model_id, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if self.h is not None and self.h.value:
            load().he_server_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulate_server(max_batch, max_wait_us, base_us, per_ct_us, arrival_us, model_of, cts_of, mem_budget=0,
                    max_inflight=0, exact_batches=False, with_refusals=False):
    """he_server_simulate_admission: the serving loop on simulated models (no GPU); mem_budget
    counts simulated ciphertexts.  Returns (batch id per request, latency ms per request), and
    with with_refusals also the refusal flag of each request."""
    n = len(arrival_us)
    opt = _lib.he_server_opts(max_batch, max_wait_us, mem_budget, max_inflight, int(exact_batches))
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    u32 = lambda a: np.ascontiguousarray(a, dtype=np.uint32)
    base, per, arr = f64(base_us), f64(per_ct_us), f64(arrival_us)
    mo, co = u32(model_of), u32(cts_of)
    batch = np.zeros(n, dtype=np.uint64)
    lat = np.zeros(n, dtype=np.float64)
    ref = np.zeros(n, dtype=np.uint32)
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    check(load().he_server_simulate_admission(ctypes.byref(opt), len(base), P(base, ctypes.c_double),
                                              P(per, ctypes.c_double), n, P(arr, ctypes.c_double),
                                              P(mo, ctypes.c_uint32), P(co, ctypes.c_uint32),
                                              P(batch, ctypes.c_uint64), P(lat, ctypes.c_double),
                                              P(ref, ctypes.c_uint32)))
    return (batch, lat, ref) if with_refusals else (batch, lat)


class Context:
    """he_context_create + key material; one CUDA stream, one device."""

    def __init__(self, logn: int, data_bits: Sequence[int], special_bits: Sequence[int], dnum: int,
                 log2_scale: float, seed: int, device: int = 0, stream: int | None = None):
        L = load()
        bits = list(data_bits) + list(special_bits)
        self._bits = (ctypes.c_uint32 * len(bits))(*bits)
        p = _lib.he_params(logn, len(data_bits), len(special_bits), self._bits, dnum, float(log2_scale), seed,
                           device, ctypes.c_void_p(stream) if stream else None)
        h = ctypes.c_void_p()
        check(L.he_context_create(ctypes.byref(p), ctypes.byref(h)))
        self.h = h
        self.logn, self.n = logn, 1 << logn
        self.n_data, self.n_special = len(data_bits), len(special_bits)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().he_context_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- context
    def primes(self):
        n = self.n_data + self.n_special
        out = (ctypes.c_uint64 * n)()
        check(load().he_context_primes(self.h, out, n))
        return list(out)

    def keygen(self, steps=()):
        arr = (ctypes.c_int32 * max(1, len(steps)))(*steps)
        check(load().he_keygen(self.h, arr, len(steps)))

    def keygen_pow2(self):
        """he_keygen_pow2: power-of-two Galois keys only; rotations by non-adjacent-form chains."""
        check(load().he_keygen_pow2(self.h))

    def set_schedule(self, schedule: str):
        """he_context_set_schedule: "fused" (the default) or "literal" (the paper's order, one
        operation at a time) for the layer calls and the models compiled from then on."""
        check(load().he_context_set_schedule(self.h, _lib.SCHEDULES[schedule]))

    def sync(self):
        check(load().he_sync(self.h))

    def launches(self) -> int:
        return int(load().he_kernel_launches(self.h))

    def profile_begin(self):
        check(load().he_profile_begin(self.h))

    def profile_end(self):
        """-> {"layer/kernel": (launches, total_ms, algorithmic_bytes, algorithmic_ops)} of the eager
        launches since profile_begin."""
        cap = 256
        buf = (_lib.he_kernel_stat * cap)()
        n = ctypes.c_size_t(0)
        check(load().he_profile_end(self.h, buf, cap, ctypes.byref(n)))
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms), float(buf[i].bytes),
                                       float(buf[i].ops)) for i in range(min(n.value, cap))}

    def ubench(self):
        """Measured register-only throughput: (butterflies/s, 128-bit MACs/s, Barrett products/s,
        SM count of the device the grids were sized for)."""
        out = (ctypes.c_double * 4)()
        check(load().he_ubench(self.h, out))
        return tuple(out)

    # ---- client side
    TUNE_KNOBS = ("ntt_split", "moddown_split", "rescale_split", "mac_group", "lazy_bt", "lazy_order", "mac_bk",
                  "mac_split", "comb_bt", "comb_fold", "mac_tc")

    def autotune(self, cache_path: str | None = None) -> dict:
        """he_autotune: time the launch-shape candidates (or read them from cache_path)."""
        import json
        buf = ctypes.create_string_buffer(8192)
        check(load().he_autotune(self.h, cache_path.encode() if cache_path else None, buf, len(buf)))
        return json.loads(buf.value.decode() or "{}")

    def tuning(self) -> dict:
        v = (ctypes.c_int32 * len(self.TUNE_KNOBS))()
        check(load().he_tuning_get(self.h, v, len(v)))
        return dict(zip(self.TUNE_KNOBS, list(v)))

    def set_tuning(self, **kw):
        cur = self.tuning()
        cur.update(kw)
        v = (ctypes.c_int32 * len(self.TUNE_KNOBS))(*[cur[k] for k in self.TUNE_KNOBS])
        check(load().he_tuning_set(self.h, v, len(v)))

    def encrypt(self, x, samples_per_ct: int, stride: int, enc_seed: int) -> Ct:
        """x: [n][H][W] (2-D), [n][C][H][W] (C channels in one ciphertext) or [n][W]
        (1-D), numpy (host) or CUDA torch tensor (device)."""
        out = ctypes.c_void_p()
        if hasattr(x, "is_cuda") and x.is_cuda:
            xs = x.contiguous()
            shape = tuple(xs.shape)
            ptr, dev = ctypes.c_void_p(xs.data_ptr()), 1
            keep = xs
        else:
            keep = np.ascontiguousarray(x, dtype=np.float64)
            shape = keep.shape
            ptr, dev = keep.ctypes.data_as(ctypes.c_void_p), 0
        if len(shape) == 2:
            n, C, H, W = shape[0], 1, 1, shape[1]
        elif len(shape) == 3:
            (n, H, W), C = shape, 1
        else:
            n, C, H, W = shape
        check(load().he_encrypt_channels(self.h, ptr, dev, C, W, H, n, samples_per_ct, stride, enc_seed,
                                         ctypes.byref(out)))
        del keep
        return Ct(self, out)

    def decrypt(self, ct: Ct, n_per_sample: int, out=None):
        """-> numpy [B*samples_per_ct][n_per_sample], or writes into a CUDA torch tensor `out`."""
        if out is not None:
            check(load().he_decrypt(self.h, ct.h, ctypes.c_void_p(out.data_ptr()), 1, n_per_sample))
            return out
        b = ct.batch
        spc = self._spc(ct)
        res = np.zeros((b * spc, n_per_sample))
        check(load().he_decrypt(self.h, ct.h, res.ctypes.data_as(ctypes.c_void_p), 0, n_per_sample))
        return res

    def _spc(self, ct):
        spc = ctypes.c_uint32()
        check(load().he_ct_layout(ct.h, ctypes.byref(spc), None, None))
        return spc.value

    def export(self, ct: Ct) -> np.ndarray:
        """Coefficient form [B][2][L'][N] (uint64)."""
        b, l, _ = ct.info()
        out = np.zeros((b, 2, l, self.n), dtype=np.uint64)
        check(load().he_ct_export(self.h, ct.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return out

    # ---- ciphertext ops
    def _one(self, fn, *args) -> Ct:
        out = ctypes.c_void_p()
        check(fn(self.h, *args, ctypes.byref(out)))
        return Ct(self, out)

    def rotate(self, ct: Ct, step: int) -> Ct:
        return self._one(load().he_rotate, ct.h, step)

    def rotate_hoisted(self, ct: Ct, steps):
        arr = (ctypes.c_int32 * len(steps))(*steps)
        outs = (ctypes.c_void_p * len(steps))()
        check(load().he_rotate_hoisted(self.h, ct.h, arr, len(steps), outs))
        return [Ct(self, outs[i]) for i in range(len(steps))]

    def rescale(self, ct: Ct) -> Ct:
        return self._one(load().he_rescale, ct.h)

    def mul_plain(self, ct: Ct, v) -> Ct:
        v = np.ascontiguousarray(v, dtype=np.float64)
        return self._one(load().he_mul_plain, ct.h, _dptr(v))

    def add(self, a: Ct, b: Ct) -> Ct:
        return self._one(load().he_add, a.h, b.h)

    def _chan(self, cts):
        arr = (ctypes.c_void_p * len(cts))(*[c.h.value for c in cts])
        return arr

    def _multi(self, n_out, fn, *args):
        outs = (ctypes.c_void_p * n_out)()
        check(fn(self.h, *args, outs))
        return [Ct(self, outs[i]) for i in range(n_out)]

    def square(self, cts):
        return self._multi(len(cts), load().he_square, self._chan(cts), len(cts))

    def pack(self, cts) -> Ct:
        """he_pack: one ciphertext carrying the samples of every input, in order."""
        return self._one(load().he_pack, self._chan(cts), len(cts))

    def drop_level(self, ct: Ct, levels: int = 1) -> Ct:
        return self._one(load().he_drop_level, ct.h, levels)

    def approx_relu(self, cts):
        return self._multi(len(cts), load().he_approx_relu, self._chan(cts), len(cts))

    def conv2d(self, cts, w, b, stride=1, incremental=False):
        w = np.ascontiguousarray(w, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        co, ci, k = w.shape[0], w.shape[1], w.shape[-1]
        return self._multi(co, load().he_conv2d, self._chan(cts), ci, _dptr(w), _dptr(b), co, k, stride,
                           int(incremental))

    def conv1d(self, cts, w, b, stride=1, incremental=False):
        w = np.ascontiguousarray(w, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        co, ci, k = w.shape
        return self._multi(co, load().he_conv1d, self._chan(cts), ci, _dptr(w), _dptr(b), co, k, stride,
                           int(incremental))

    def avgpool(self, cts, c: int):
        return self._multi(len(cts), load().he_avgpool, self._chan(cts), len(cts), c)

    def flatten(self, cts) -> Ct:
        return self._one(load().he_flatten, self._chan(cts), len(cts))

    def fc(self, ct: Ct, W, b) -> Ct:
        W = np.ascontiguousarray(W, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        dout, din = W.shape
        return self._one(load().he_fc, ct.h, _dptr(W), _dptr(b), din, dout)

    def compile(self, layers, W_img: int, H_img: int, samples_per_ct: int) -> Model:
        arr, keep = layers_to_c(layers)
        h = ctypes.c_void_p()
        check(load().he_model_compile(self.h, arr, len(layers), W_img, H_img, samples_per_ct, ctypes.byref(h)))
        return Model(self, h, keep)

    def ntt(self, data_ptr: int, n_limbs: int, prime_idx, inverse: bool = False):
        arr = (ctypes.c_uint32 * n_limbs)(*prime_idx)
        check(load().he_ntt(self.h, ctypes.c_void_p(data_ptr), n_limbs, arr, int(inverse)))
