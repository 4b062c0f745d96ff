"""The serving loop's scheduling on simulated models (no GPU): the same C++
loop as the GPU server, with batches that occupy a simulated device for a
modelled time.  Checks continuous batching, FIFO order per model, the batch
size bound, round-robin service across models and the latency bookkeeping."""
import numpy as np
import pytest

lib = pytest.importorskip("paper_2402_03060_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_03060_gb300 import build
    build.build()


def poisson(rate_per_s, n, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1e6 / rate_per_s, n))


def check_fifo(batch, model_of, cts_of, max_batch):
    for m in set(model_of.tolist()):
        idx = np.nonzero(model_of == m)[0]
        b = batch[idx]
        assert np.all(np.diff(b.astype(np.int64)) >= 0), "requests of one model served out of order"
    for bid in set(batch.tolist()):
        idx = np.nonzero(batch == bid)[0]
        assert len(set(model_of[idx].tolist())) == 1, "a batch mixes models"
        assert cts_of[idx].sum() <= max_batch


def test_light_load_runs_each_request_alone():
    # arrivals 20 ms apart, batches take 2 ms: no queueing, latency = service time
    n = 12
    arr = np.arange(n) * 40000.0
    mo = np.zeros(n, np.uint32)
    co = np.ones(n, np.uint32)
    batch, lat = lib.simulate_server(8, 0, [2000.0], [0.0], arr, mo, co)
    assert len(set(batch.tolist())) == n
    assert np.all(lat >= 1.9) and np.median(lat) < 20.0


def test_burst_fills_batches_in_arrival_order():
    # 40 requests at once for one model, 8 per batch, 10 ms per batch
    n = 40
    arr = np.zeros(n)
    mo = np.zeros(n, np.uint32)
    co = np.ones(n, np.uint32)
    batch, lat = lib.simulate_server(8, 0, [10000.0], [0.0], arr, mo, co)
    check_fifo(batch, mo, co, 8)
    sizes = np.bincount(batch.astype(np.int64))[1:]
    sizes = sizes[sizes > 0]
    # the first two batches launch at once with what has arrived (two may be in flight);
    # from then on the queue is long and batches are full
    assert sizes.sum() == n and sizes.max() == 8
    assert len(sizes) <= n // 8 + 2 and (sizes == 8).sum() >= n // 8 - 2
    # latency grows by one batch time per batch ahead (two batches may be queued on the device)
    assert lat.max() < 10.0 * (len(sizes) + 1) + 20.0


def test_continuous_batching_joins_running_model():
    # a long batch is running; requests arriving meanwhile form the next batch together
    arr = np.array([0.0, 5000, 10000, 15000, 20000, 25000])
    mo = np.zeros(6, np.uint32)
    co = np.ones(6, np.uint32)
    batch, _ = lib.simulate_server(4, 400000, [300000.0], [0.0], arr, mo, co)
    check_fifo(batch, mo, co, 4)
    assert batch[0] != batch[1]
    assert len(set(batch[1:5].tolist())) == 1      # four arrivals during the first batch: one full batch


def test_mixed_models_and_sizes():
    n = 300
    rng = np.random.default_rng(12345)
    arr = poisson(2000.0, n, 12345)
    mo = rng.integers(0, 3, n).astype(np.uint32)
    co = rng.integers(1, 3, n).astype(np.uint32)
    base = [300.0, 900.0, 200.0]
    per = [40.0, 120.0, 30.0]
    batch, lat = lib.simulate_server(8, 0, base, per, arr, mo, co)
    check_fifo(batch, mo, co, 8)
    assert np.all(lat > 0)
    # every model got served while the others were busy (no starvation)
    for m in range(3):
        assert np.all(batch[mo == m] > 0)


def test_invalid_trace_is_rejected():
    with pytest.raises(lib.HeError):
        lib.simulate_server(4, 0, [100.0], [0.0], [0.0, 10.0], np.array([0, 3], np.uint32), np.ones(2, np.uint32))
    with pytest.raises(lib.HeError):
        lib.simulate_server(4, 0, [100.0], [0.0], [0.0], np.zeros(1, np.uint32), np.array([5], np.uint32))


def test_one_batch_in_flight_and_exact_batches_cut_latency():
    """Near capacity (a batch of b costs 1 ms + 1 ms per ciphertext of its bucket; 800
    requests/s against about 890/s with full batches), one batch in flight per model
    lets the queue fill the next batch while one runs, and exact batch sizes stop
    paying for power-of-two padding: lower median and tail latency than the padded,
    two-in-flight policy."""
    n = 600
    arr = poisson(800.0, n, 7)
    mo = np.zeros(n, np.uint32)
    co = np.ones(n, np.uint32)
    b2, lat2 = lib.simulate_server(8, 0, [1000.0], [1000.0], arr, mo, co)
    b1, lat1 = lib.simulate_server(8, 0, [1000.0], [1000.0], arr, mo, co, max_inflight=1, exact_batches=True)
    check_fifo(b1, mo, co, 8)
    assert np.median(lat1) < 0.8 * np.median(lat2)
    assert np.percentile(lat1, 99) < np.percentile(lat2, 99)


def test_memory_admission_refuses_then_admits_in_order():
    """mem_budget holds exactly k = 3 request ciphertexts: of six one-ciphertext requests
    arriving at once, the first three are admitted and run as one batch; the other three
    are refused on arrival and admitted, in arrival order, once that batch completes."""
    n, k = 6, 3
    arr = np.zeros(n)
    mo = np.zeros(n, np.uint32)
    co = np.ones(n, np.uint32)
    batch, lat, ref = lib.simulate_server(8, 0, [20000.0], [0.0], arr, mo, co, mem_budget=k, max_inflight=1,
                                          with_refusals=True)
    assert ref.tolist() == [0, 0, 0, 1, 1, 1]
    check_fifo(batch, mo, co, 8)
    assert len(set(batch[:k].tolist())) == 1 and len(set(batch[k:].tolist())) == 1
    assert batch[k] > batch[0]
    # the refused ones waited for the first batch: about two batch times from their arrival
    assert np.all(lat[:k] < 35.0) and np.all(lat[k:] >= 39.0) and np.all(lat[k:] < 80.0)


def test_memory_admission_unlimited_and_multi_ciphertext_requests():
    """Without a budget nothing is refused; a two-ciphertext request needs room for both."""
    arr = np.array([0.0, 0.0, 0.0, 1000.0])
    mo = np.zeros(4, np.uint32)
    co = np.array([1, 1, 2, 1], np.uint32)
    _, _, ref = lib.simulate_server(8, 0, [10000.0], [0.0], arr, mo, co, with_refusals=True)
    assert ref.tolist() == [0, 0, 0, 0]
    # budget 3: requests 0 and 1 fit (2 cts), request 2 (2 cts) does not, request 3 queues behind it
    batch, lat, ref = lib.simulate_server(8, 0, [10000.0], [0.0], arr, mo, co, mem_budget=3, max_inflight=1,
                                          with_refusals=True)
    assert ref.tolist() == [0, 0, 1, 1]
    check_fifo(batch, mo, co, 8)
