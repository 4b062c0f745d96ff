// server.cu -- continuous-batching serving loop over compiled models.
//
// The paper's service model: clients encrypt their inputs with the public key,
// the server evaluates the network on the ciphertexts with the evaluation keys
// and returns encrypted results.  This loop serves several compiled models
// (possibly on different contexts and ring degrees) from one host thread:
//   * each model has a FIFO queue; a request is one ciphertext batch (he_ct);
//   * whenever a model has fewer than max_inflight batches in flight (2 by
//     default), the worker takes the queued requests in arrival order, as many as
//     fit in max_batch ciphertexts, gathers them into one batch -- padded to a
//     power of two (a model sees at most log2(max_batch)+1 batch shapes) or, with
//     exact_batches, of its own size -- replayed from that shape's CUDA graph, and
//     launches it on the model's stream; requests that arrive while a batch runs
//     join the next one (continuous batching);
//   * completion is signalled from the stream (cudaLaunchHostFunc), the result
//     batch is split into per-request views, and waiting clients are woken;
//   * admission: a model is accepted only if the device bytes it holds (keys,
//     cached masks, graph pools) fit the memory budget, and a request only if
//     the budget still holds its ciphertext bytes from submission until its
//     result is collected (queued, running, or finished and not yet collected);
//     a refused request gets HE_ENOMEM and may be submitted again once results
//     have been collected.
// Every ciphertext's result is independent of the batch it ran in (all kernels
// act per ciphertext), so a request's output is bit-identical alone or mixed.
//
// Locking: srv->mu guards the queues and is a leaf lock (no CUDA call and no
// context lock is taken while it is held); a context's lock is taken only by
// the worker while it gathers/launches or splits a batch of that context.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>

#include "model.cuh"

using SrvClock = std::chrono::steady_clock;

namespace {

struct Request {
    u64 id = 0;
    u32 model = 0, B = 0;
    Cts in;                                   // shares the caller's buffer
    SrvClock::time_point t_submit, t_done;
    int state = 0;                            // 0 queued, 1 running, 2 done
    he_status err = HE_OK;
    std::string msg;
    he_ct *out = nullptr;
    u64 batch = 0;
    size_t bytes = 0;
};

struct Model;
struct Batch {
    he_server *srv = nullptr;
    Model *M = nullptr;
    u64 id = 0;
    u32 model = 0, bucket = 0;
    std::vector<Request *> reqs;
    Cts out;
    SrvClock::time_point t_done;
    he_status err = HE_OK;
    std::string msg;
    double sim_us = 0;
};

struct Model {
    he_model *m = nullptr;                    // nullptr: simulated model
    std::deque<Request *> q;
    u32 inflight = 0;
    double sim_base_us = 0, sim_per_ct_us = 0;
    std::vector<double> lat_ms;
    u64 batches = 0, cts = 0, requests = 0;
    size_t resident = 0;
};

u32 pow2_at_least(u32 v) {
    u32 p = 1;
    while (p < v) p <<= 1;
    return p;
}
u32 pow2_at_most(u32 v) {
    u32 p = 1;
    while (p * 2 <= v) p <<= 1;
    return p;
}

}  // namespace

struct he_server {
    he_server_opts opt;
    bool simulate = false;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::unique_ptr<Model>> models;   // grows under mu; a Model never moves
    std::map<u64, Request *> reqs;
    std::deque<Batch *> done;
    u64 next_req = 1, next_batch = 1;
    u32 rr = 0, inflight = 0;
    size_t resident = 0, pending = 0;         // bytes: models' holdings; requests submitted, not yet collected
    std::vector<Ctx *> counted;               // contexts whose pools are already in `resident`
    bool stop = false;
    std::thread worker;
    // simulated device: one queue of batches run back to back
    std::mutex sim_mu;
    std::condition_variable sim_cv;
    std::deque<Batch *> sim_q;
    bool sim_stop = false;
    std::thread sim_thread;
};

static void CUDART_CB batch_done(void *p) {
    Batch *b = static_cast<Batch *>(p);
    he_server *s = b->srv;
    b->t_done = SrvClock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    s->done.push_back(b);
    s->cv.notify_all();
}

static void sim_loop(he_server *s) {
    std::unique_lock<std::mutex> lk(s->sim_mu);
    while (true) {
        s->sim_cv.wait(lk, [&] { return s->sim_stop || !s->sim_q.empty(); });
        if (s->sim_q.empty()) return;
        Batch *b = s->sim_q.front();
        s->sim_q.pop_front();
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds((long long)b->sim_us));
        batch_done(b);
        lk.lock();
    }
}

// gather the batch, run the model, signal completion from the stream
static void launch_batch(he_server *s, Batch *b) {
    Model &M = *b->M;
    if (s->simulate) {
        b->sim_us = M.sim_base_us + M.sim_per_ct_us * b->bucket;
        std::lock_guard<std::mutex> lk(s->sim_mu);
        s->sim_q.push_back(b);
        s->sim_cv.notify_all();
        return;
    }
    he_model *m = M.m;
    Ctx *c = m->c;
    try {
        CtxLock lk(c);
        CUDA_TRY(cudaSetDevice(c->device));
        const Cts &x0 = b->reqs[0]->in;
        const size_t cw = cts_ct_words(c, x0.lp);
        Cts x = cts_alloc(c, b->bucket, x0.lp, x0.scale, x0.lay);
        size_t at = 0;
        for (Request *r : b->reqs) {
            CUDA_TRY(cudaMemcpyAsync(x.data() + at * cw, r->in.data(), r->B * cw * 8, cudaMemcpyDeviceToDevice,
                                     c->stream));
            at += r->B;
        }
        for (; at < b->bucket; ++at)   // padding: copies of the first ciphertext, results discarded
            CUDA_TRY(cudaMemcpyAsync(x.data() + at * cw, x0.data(), cw * 8, cudaMemcpyDeviceToDevice, c->stream));
        b->out = model_infer(m, x, true);
        CUDA_TRY(cudaLaunchHostFunc(c->stream, batch_done, b));
    } catch (const HeError &e) {
        b->err = e.code;
        b->msg = e.what();
        batch_done(b);
    } catch (const std::exception &e) {
        b->err = HE_EINVAL;
        b->msg = e.what();
        batch_done(b);
    }
}

// split the result batch into per-request handles and drop the inputs
static void retire_batch(he_server *s, Batch *b) {
    if (s->simulate) return;
    Ctx *c = b->M->m->c;
    CtxLock lk(c);
    // each request's slice of the result batch, in the result's own ciphertext size
    const size_t cw = cts_ct_words(c, b->out.lp);
    size_t at = 0;
    for (Request *r : b->reqs) {
        if (b->err == HE_OK) r->out = ct_wrap(c, cts_view(b->out, at * cw, r->B));
        at += r->B;
        r->in = Cts();
    }
    b->out = Cts();
}

static void server_loop(he_server *s) {
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        while (!s->done.empty()) {
            Batch *b = s->done.front();
            s->done.pop_front();
            lk.unlock();
            retire_batch(s, b);
            lk.lock();
            Model &M = *b->M;
            M.inflight--;
            s->inflight--;
            M.batches++;
            M.cts += b->bucket;
            for (Request *r : b->reqs) {
                r->state = 2;
                r->err = b->err;
                r->msg = b->msg;
                r->t_done = b->t_done;
                if (s->simulate) s->pending -= r->bytes;   // simulated requests are collected on completion
                M.requests++;
                M.lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
            }
            delete b;
            s->cv.notify_all();
        }
        bool queued = false;
        for (auto &M : s->models) queued |= !M->q.empty();
        if (s->stop && !queued && s->inflight == 0) return;
        bool launched = false;
        SrvClock::time_point wake = SrvClock::now() + std::chrono::milliseconds(50);
        const u32 nm = (u32)s->models.size();
        for (u32 k = 0; k < nm; ++k) {
            const u32 mi = (s->rr + k) % nm;
            Model &M = *s->models[mi];
            if (M.q.empty() || M.inflight >= s->opt.max_inflight) continue;
            u32 total = 0;
            for (Request *r : M.q) {
                if (total + r->B > s->opt.max_batch) break;
                total += r->B;
            }
            if (s->opt.max_wait_us && total < s->opt.max_batch && M.inflight > 0 && !s->stop) {
                // a batch is running: hold a partial batch until it fills or its oldest request waited max_wait_us
                auto due = M.q.front()->t_submit + std::chrono::microseconds(s->opt.max_wait_us);
                if (SrvClock::now() < due) {
                    wake = std::min(wake, due);
                    continue;
                }
            }
            Batch *b = new Batch();
            b->srv = s;
            b->M = &M;
            b->id = s->next_batch++;
            b->model = mi;
            u32 got = 0;
            while (!M.q.empty() && got + M.q.front()->B <= s->opt.max_batch) {
                Request *r = M.q.front();
                M.q.pop_front();
                r->state = 1;
                r->batch = b->id;
                got += r->B;
                b->reqs.push_back(r);
            }
            b->bucket = s->opt.exact_batches ? got : pow2_at_least(got);   // <= max_batch
            M.inflight++;
            s->inflight++;
            s->rr = mi + 1;
            launched = true;
            lk.unlock();
            launch_batch(s, b);
            lk.lock();
        }
        if (!launched && s->done.empty()) s->cv.wait_until(lk, wake);
    }
}

// whether the budget holds `bytes` more of requests (caller holds s->mu)
static bool admits(const he_server *s, size_t bytes) {
    return !s->opt.mem_budget || s->resident + s->pending + bytes <= s->opt.mem_budget;
}

static size_t model_bytes(const he_model *m) {
    return m->gpool.bytes_live + m->gpool.bytes_cached;
}

// ------------------------------------------------------------------ C ABI
const char *set_last_error(const char *msg);

template <class F>
static he_status srv_guard(F &&f) {
    try {
        f();
        return HE_OK;
    } catch (const HeError &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return HE_EINVAL;
    }
}

static void start_threads(he_server *s) {
    s->worker = std::thread(server_loop, s);
    if (s->simulate) s->sim_thread = std::thread(sim_loop, s);
}

// max_batch rounded down to a power of two; max_inflight 0 -> 2
static he_server_opts normalized(he_server_opts o) {
    o.max_batch = pow2_at_most(o.max_batch);
    if (!o.max_inflight) o.max_inflight = 2;
    o.exact_batches = o.exact_batches ? 1 : 0;
    return o;
}

extern "C" {

he_status he_server_create(const he_server_opts *opt, he_server **out) {
    return srv_guard([&] {
        if (!opt || !out || opt->max_batch < 1) throw HeError(HE_EINVAL, "bad server options");
        he_server *s = new he_server();
        s->opt = normalized(*opt);
        start_threads(s);
        *out = s;
    });
}

he_status he_server_add_model(he_server *s, he_model *m, uint32_t *model_id) {
    return srv_guard([&] {
        if (!s || !m || !model_id || s->simulate) throw HeError(HE_EINVAL, "bad arguments");
        Ctx *c = m->c;
        size_t held = 0;
        {
            // warm every batch shape the loop can launch: captures its CUDA graph and sizes its pool
            CtxLock lk(c);
            CUDA_TRY(cudaSetDevice(c->device));
            const u32 lp = c->L1;
            Layout L;
            L.W_img = m->W_img;
            L.H_img = m->H_img;
            L.W = m->W_img;
            L.H = m->H_img;
            L.stride = m->plan.stride;
            L.n_samples = m->spc;
            L.dims = m->H_img == 1 ? 1 : 2;
            // largest shape first: the smaller shapes' captures reuse its buffers in the model's graph pool
            for (u32 b = s->opt.max_batch; b >= 1; b = s->opt.exact_batches ? b - 1 : b >> 1) {
                Cts x = cts_alloc(c, b, lp, c->scale, L);
                CUDA_TRY(cudaMemsetAsync(x.data(), 0, (size_t)b * cts_ct_words(c, lp) * 8, c->stream));
                Cts y = model_infer(m, x, true);
            }
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            held = model_bytes(m);
        }
        std::lock_guard<std::mutex> lk(s->mu);
        size_t add = held;
        if (std::find(s->counted.begin(), s->counted.end(), c) == s->counted.end())
            add += c->pool.bytes_live + c->pool.bytes_cached;
        if (s->opt.mem_budget && s->resident + add > s->opt.mem_budget)
            throw HeError(HE_ENOMEM, fmt("model needs %zu device bytes; %zu of the %llu-byte budget are held",
                                         add, s->resident, (unsigned long long)s->opt.mem_budget));
        if (std::find(s->counted.begin(), s->counted.end(), c) == s->counted.end()) s->counted.push_back(c);
        s->resident += add;
        std::unique_ptr<Model> M(new Model());
        M->m = m;
        M->resident = add;
        s->models.push_back(std::move(M));
        *model_id = (uint32_t)s->models.size() - 1;
    });
}

he_status he_server_submit(he_server *s, uint32_t model_id, const he_ct *in, uint64_t *req_id) {
    return srv_guard([&] {
        if (!s || !in || !req_id) throw HeError(HE_EINVAL, "bad arguments");
        std::lock_guard<std::mutex> lk(s->mu);
        if (model_id >= s->models.size() || s->stop) throw HeError(HE_EINVAL, "unknown model or server stopping");
        Model &M = *s->models[model_id];
        if (in->x.B > s->opt.max_batch) throw HeError(HE_EINVAL, "request larger than max_batch ciphertexts");
        if (in->c != M.m->c) throw HeError(HE_EINVAL, "ciphertext belongs to another context");
        model_check_input(M.m, in->x);
        const size_t bytes = (size_t)in->x.B * cts_ct_words(in->c, in->x.lp) * 8;
        if (!admits(s, bytes))
            throw HeError(HE_ENOMEM, "admission refused: the memory budget is held by requests not yet collected");
        Request *r = new Request();
        r->id = s->next_req++;
        r->model = model_id;
        r->B = in->x.B;
        r->in = in->x;
        r->bytes = bytes;
        r->t_submit = SrvClock::now();
        s->pending += bytes;
        s->reqs[r->id] = r;
        M.q.push_back(r);
        *req_id = r->id;
        s->cv.notify_all();
    });
}

he_status he_server_wait(he_server *s, uint64_t req_id, uint32_t timeout_ms, he_ct **out, double *latency_ms) {
    return srv_guard([&] {
        if (!s) throw HeError(HE_EINVAL, "null server");
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->reqs.find(req_id);
        if (it == s->reqs.end()) throw HeError(HE_EINVAL, "unknown request id");
        Request *r = it->second;
        if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->state == 2; }))
            throw HeError(HE_ETIMEOUT, "request not finished within the timeout");
        s->reqs.erase(it);
        s->pending -= r->bytes;   // collected: its bytes leave the budget
        s->cv.notify_all();
        lk.unlock();
        const he_status err = r->err;
        const std::string msg = r->msg;
        if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
        if (err == HE_OK) {
            if (out)
                *out = r->out;
            else if (r->out)
                he_ct_free(r->out);
        }
        delete r;
        if (err != HE_OK) throw HeError(err, msg);
    });
}

he_status he_server_poll(he_server *s, uint64_t req_id, int *done) {
    return srv_guard([&] {
        if (!s || !done) throw HeError(HE_EINVAL, "bad arguments");
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(req_id);
        if (it == s->reqs.end()) throw HeError(HE_EINVAL, "unknown request id");
        *done = it->second->state == 2 ? 1 : 0;
    });
}

he_status he_server_stats_get(he_server *s, int32_t model_id, he_server_stats *out) {
    return srv_guard([&] {
        if (!s || !out) throw HeError(HE_EINVAL, "bad arguments");
        std::lock_guard<std::mutex> lk(s->mu);
        std::vector<double> lat;
        he_server_stats st = {};
        for (size_t i = 0; i < s->models.size(); ++i) {
            if (model_id >= 0 && (size_t)model_id != i) continue;
            const Model &M = *s->models[i];
            lat.insert(lat.end(), M.lat_ms.begin(), M.lat_ms.end());
            st.requests += M.requests;
            st.batches += M.batches;
            st.cts += M.cts;
        }
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double p) {
            if (lat.empty()) return 0.0;
            size_t k = (size_t)std::ceil(p * lat.size());   // nearest-rank percentile
            return lat[std::min(lat.size() - 1, k ? k - 1 : 0)];
        };
        st.mean_batch = st.batches ? (double)st.cts / st.batches : 0.0;
        st.p50_ms = pct(0.50);
        st.p99_ms = pct(0.99);
        st.max_ms = lat.empty() ? 0.0 : lat.back();
        st.resident_bytes = s->resident;
        *out = st;
    });
}

void he_server_destroy(he_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    s->worker.join();   // drains: queued requests still run
    if (s->simulate) {
        {
            std::lock_guard<std::mutex> lk(s->sim_mu);
            s->sim_stop = true;
            s->sim_cv.notify_all();
        }
        s->sim_thread.join();
    }
    for (auto &kv : s->reqs) {
        if (kv.second->out) he_ct_free(kv.second->out);
        if (kv.second->in.mem) {
            std::shared_ptr<Ctx> k = s->models[kv.second->model]->m->keep;
            CtxLock lk(k.get());
            kv.second->in = Cts();
        }
        delete kv.second;
    }
    delete s;
}

// Replays an arrival trace through the same loop with simulated models: a
// batch of b ciphertexts of model i "runs" for base_us[i] + per_ct_us[i]*b on
// one simulated device (batches back to back).  No GPU is used.
he_status he_server_simulate(const he_server_opts *opt, uint32_t n_models, const double *base_us,
                             const double *per_ct_us, size_t n_req, const double *arrival_us,
                             const uint32_t *model_of, const uint32_t *cts_of, uint64_t *batch_of,
                             double *latency_ms) {
    return he_server_simulate_admission(opt, n_models, base_us, per_ct_us, n_req, arrival_us, model_of, cts_of,
                                        batch_of, latency_ms, nullptr);
}

he_status he_server_simulate_admission(const he_server_opts *opt, uint32_t n_models, const double *base_us,
                                       const double *per_ct_us, size_t n_req, const double *arrival_us,
                                       const uint32_t *model_of, const uint32_t *cts_of, uint64_t *batch_of,
                                       double *latency_ms, uint32_t *refusals) {
    return srv_guard([&] {
        if (!opt || !n_models || !base_us || !per_ct_us || (n_req && (!arrival_us || !model_of || !cts_of)) ||
            opt->max_batch < 1)
            throw HeError(HE_EINVAL, "bad arguments");
        he_server *s = new he_server();
        s->opt = normalized(*opt);
        s->simulate = true;
        for (u32 i = 0; i < n_models; ++i) {
            std::unique_ptr<Model> M(new Model());
            M->sim_base_us = base_us[i];
            M->sim_per_ct_us = per_ct_us[i];
            s->models.push_back(std::move(M));
        }
        start_threads(s);
        std::vector<Request *> all(n_req, nullptr);
        std::vector<uint32_t> refused(n_req, 0);   // 1: refused on arrival, admitted later
        std::deque<size_t> blocked;   // refused requests, retried in arrival order as the budget frees
        const auto t0 = SrvClock::now();
        he_status bad = HE_OK;
        // admit request k if the budget holds it (one simulated ciphertext counts as one byte;
        // the simulated models hold none); the latency counts from its first submission
        auto try_admit = [&](size_t k, SrvClock::time_point first) {
            const size_t bytes = cts_of[k];
            if (!admits(s, bytes)) return false;
            Request *r = new Request();
            r->id = s->next_req++;
            r->model = model_of[k];
            r->B = cts_of[k];
            r->bytes = bytes;
            r->t_submit = first;
            s->pending += bytes;
            all[k] = r;
            s->models[r->model]->q.push_back(r);
            s->cv.notify_all();
            return true;
        };
        std::vector<SrvClock::time_point> first(n_req);
        auto retry_blocked = [&] {
            while (!blocked.empty() && try_admit(blocked.front(), first[blocked.front()])) blocked.pop_front();
        };
        for (size_t k = 0; k < n_req; ++k) {
            const auto due = t0 + std::chrono::microseconds((long long)arrival_us[k]);
            std::unique_lock<std::mutex> lk(s->mu);
            // until request k is due, admit refused ones whenever a completion frees the budget
            while (!blocked.empty() && SrvClock::now() < due) {
                retry_blocked();
                if (!blocked.empty()) s->cv.wait_until(lk, due);
            }
            lk.unlock();
            std::this_thread::sleep_until(due);
            lk.lock();
            if (model_of[k] >= n_models || cts_of[k] < 1 || cts_of[k] > s->opt.max_batch) {
                bad = HE_EINVAL;
                break;
            }
            first[k] = SrvClock::now();
            retry_blocked();
            if (!blocked.empty() || !try_admit(k, first[k])) {   // FIFO: behind the refused ones
                refused[k] = 1;
                blocked.push_back(k);
            }
        }
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                if (bad == HE_OK) retry_blocked();
                if (bad == HE_OK && !blocked.empty()) return false;
                for (Request *r : all)
                    if (r && r->state != 2) return false;
                return true;
            });
        }
        for (size_t k = 0; k < n_req; ++k) {
            if (!all[k]) continue;
            if (batch_of) batch_of[k] = all[k]->batch;
            if (refusals) refusals[k] = refused[k];
            if (latency_ms)
                latency_ms[k] = std::chrono::duration<double, std::milli>(all[k]->t_done - all[k]->t_submit).count();
            delete all[k];
        }
        he_server_destroy(s);
        if (bad != HE_OK) throw HeError(bad, "bad request in the trace");
    });
}

}  // extern "C"
