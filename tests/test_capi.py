"""CPU checks of the C ABI: the library loads, exports every entry point the
header declares, and its host-side planner (he_model_plan, no GPU needed)
agrees with the oracle's planner."""
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import layers as olayers

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "unihenn.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2402_03060_gb300 import build
    build.build()
    import paper_2402_03060_gb300 as G
    return G


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(he_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ["he_keygen", "he_encrypt", "he_conv2d", "he_conv1d", "he_avgpool", "he_fc", "he_square",
              "he_decrypt", "he_flatten", "he_infer"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import subprocess
    from paper_2402_03060_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (he_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # and the binding declares each of them with the same name
    assert set(declared_functions()) <= set(_lib.SIGNATURES)
    L = lib.load()
    for n in declared_functions():
        assert hasattr(L, n)


@pytest.mark.parametrize("name", ["lenet1", "cnn1d", "cnn1d_tree", "lenet5", "m3", "conv", "M1", "M4", "M5", "m5n",
                                  "M6", "M7"])
def test_planner_matches_oracle(lib, name):
    if name in W.PAPER_MODELS:
        model, Wi, Hi = W.paper_model(name)
    elif name == "m5n":
        model, Wi, Hi = W.m5_narrow(), 32, 32
    elif name == "lenet1":
        model, Wi, Hi = W.lenet1(), 28, 28
    elif name == "m3":
        model, Wi, Hi = W.m3_relu(), 28, 28
    elif name == "cnn1d":
        model, Wi, Hi = W.cnn1d(), 1024, 1
    elif name == "cnn1d_tree":
        model, Wi, Hi = W.cnn1d(fc_sum="tree"), 1024, 1
    elif name == "lenet5":
        model, Wi, Hi = W.lenet5_sq(), 32, 32
    else:
        model, Wi, Hi = W.single_conv(), 28, 28
    stride, levels, steps = lib.plan(model, Wi, Hi)
    p = olayers.plan(model, Wi, Hi, 1 if Hi == 1 else 2)
    assert stride == p["stride"] and levels == p["levels"] and steps == p["steps"]


@pytest.mark.parametrize("co", [16, 17])
def test_planner_flatten_merge_boundary(lib, co):
    """The flatten's last masked stage (8 rows) is merged with the packing of co channels
    when 8*co <= 128 rotation steps: both planners agree on either side of the bound."""
    rng = np.random.default_rng(co)
    model = [{"op": "conv2d", "w": rng.normal(0, 0.1, (co, 1, 5, 5)), "b": np.zeros(co), "stride": 1},
             {"op": "square"}, {"op": "avgpool", "k": 3}, {"op": "flatten"},
             {"op": "fc", "w": rng.normal(0, 0.1, (10, co * 64)), "b": np.zeros(10)}]
    stride, levels, steps = lib.plan(model, 28, 28)
    p = olayers.plan(model, 28, 28, 2)
    assert stride == p["stride"] and levels == p["levels"] and steps == p["steps"]
    rows = {r * (28 * 3 - 8) for r in range(8)}            # the last stage: 8 rows
    merged = {s - o * 64 for s in rows for o in range(co)} - {0}
    probe = 7 * 76 - 15 * 64                               # row 7 of channel 15: a merged step only
    if 8 * co <= olayers.MERGE_MAX_STEPS:
        assert merged <= set(steps) and probe in steps     # rows x channels, one combination
    else:
        assert rows - {0} <= set(steps) and {-o * 64 for o in range(1, co)} <= set(steps)
        assert probe not in steps


def test_planner_rejects_bad_models(lib):
    from paper_2402_03060_gb300 import HeError
    bad = [{"op": "conv2d", "w": np.zeros((1, 1, 30, 30)), "b": np.zeros(1), "stride": 1}]
    with pytest.raises(HeError) as e:
        lib.plan(bad, 28, 28)
    assert e.value.status == 1
    bad_fc = W.lenet1()[:-1] + [{"op": "fc", "w": np.zeros((10, 100)), "b": np.zeros(10)}]
    with pytest.raises(HeError):
        lib.plan(bad_fc, 28, 28)
    conv2d_on_signal = [{"op": "conv2d", "w": np.zeros((1, 1, 3, 3)), "b": np.zeros(1), "stride": 1}]
    with pytest.raises(HeError):
        lib.plan(conv2d_on_signal, 64, 1)
    channels_on_signal = [{"op": "conv1d", "w": np.zeros((2, 3, 3)), "b": np.zeros(2), "stride": 1}]
    with pytest.raises(HeError):
        lib.plan(channels_on_signal, 64, 1)      # several input channels need a 2-D image
    big_pool = [{"op": "conv2d", "w": np.zeros((1, 1, 3, 3)), "b": np.zeros(1), "stride": 1},
                {"op": "avgpool", "k": 30}]
    with pytest.raises(HeError):
        lib.plan(big_pool, 28, 28)
    fc_first = [{"op": "fc", "w": np.zeros((10, 784)), "b": np.zeros(10)}]
    with pytest.raises(HeError):
        lib.plan(fc_first, 28, 28)               # FC needs a flattened input


@pytest.mark.parametrize("case", ["1d_pool_merged", "1d_pool_separate", "conv_two_stages_separate"])
def test_planner_flatten_variants(lib, case):
    rng = np.random.default_rng(7)
    if case.startswith("1d"):
        co = 4 if case.endswith("merged") else 40
        model = [{"op": "conv1d", "w": rng.normal(0, 0.1, (co, 1, 3)), "b": rng.normal(0, 0.1, co), "stride": 1},
                 {"op": "square"}, {"op": "avgpool", "k": 2}, {"op": "flatten"},
                 {"op": "fc", "w": rng.normal(0, 0.1, (5, co * 31)), "b": rng.normal(0, 0.1, 5)}]
        Wi, Hi = 64, 1
    else:
        model = [{"op": "conv2d", "w": rng.normal(0, 0.1, (17, 1, 4, 4)), "b": rng.normal(0, 0.1, 17), "stride": 3},
                 {"op": "square"}, {"op": "flatten"},
                 {"op": "fc", "w": rng.normal(0, 0.1, (10, 17 * 81)), "b": rng.normal(0, 0.1, 10)}]
        Wi, Hi = 28, 28
    stride, levels, steps = lib.plan(model, Wi, Hi)
    p = olayers.plan(model, Wi, Hi, 1 if Hi == 1 else 2)
    assert stride == p["stride"] and levels == p["levels"] and steps == p["steps"]


_NULL_CALLS = r'''
import ctypes, json, sys
sys.path.insert(0, sys.argv[1])
from paper_2402_03060_gb300 import _lib
L = _lib.load()
out = {}
for name, (res, args) in sorted(_lib.SIGNATURES.items()):
    vals = [0.0 if a is ctypes.c_double else
            0 if a in (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int, ctypes.c_size_t) else None
            for a in args]
    r = getattr(L, name)(*vals)
    out[name] = r if isinstance(r, int) or r is None else repr(r)
print(json.dumps(out))
'''


def test_every_entry_point_refuses_null_arguments(lib):
    """Each call of the C ABI with null handles and pointers and zero sizes returns HE_EINVAL (the
    void teardown calls return, the counters read 0) and crashes nothing -- no GPU needed: the
    arguments are checked before any device work.  Run in a child process."""
    import json
    import subprocess
    import sys
    from paper_2402_03060_gb300 import _lib
    p = subprocess.run([sys.executable, "-c", _NULL_CALLS, ROOT], capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    got = json.loads(p.stdout.strip().splitlines()[-1])
    assert set(got) == set(_lib.SIGNATURES)
    for name, r in got.items():
        if name in ("he_context_destroy", "he_ct_free", "he_model_free", "he_server_destroy"):
            assert r is None, name
        elif name == "he_kernel_launches":
            assert r == 0
        elif name == "he_last_error":
            continue
        else:
            assert r == _lib.HE_EINVAL, (name, r)
