// rambo_server.cu -- continuous-batching query server over graph-captured
// plans, with streaming set inserts (Sec. 3.1: RAMBO takes updates from a
// stream).
//
// One worker thread owns the GPU side.  Requests (key queries, sequence
// queries, insert batches) are copied into host queues by rambo_server_submit*.
// The worker keeps up to `slots` plans per query kind in flight, each on its
// own stream: whenever a slot is free it takes every queued query of that
// kind that fits the slot's buffers (admission by device memory), copies them
// into the slot's pinned staging, and replays the slot's captured graph.  New
// requests are admitted while other batches run, so their work overlaps on
// the device.  An insert is an ordering barrier: queries submitted before it
// finish first and see the old index; queries submitted after it wait for it
// and see the new index.  A query's answer depends only on the index state at
// its turn, never on which batch it rode in.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rambo_impl.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Op {
    uint64_t ticket = 0;
    uint64_t seq = 0;  // submission order
    int type = 0;      // 0 query, 1 insert
    int kind = 1;      // 0 keys, 1 DNA
    std::vector<uint8_t> data;
    uint64_t items = 0;  // keys or bases
    std::vector<uint64_t> set_ids, offsets;
    uint32_t k = 31;
    bool solo = false;  // results overflowed a shared batch: run alone
    uint32_t deferrals = 0;  // times its batch was deferred for want of pinned memory
    Clock::time_point t_submit;
};

// A query whose batch could not get pinned memory for its answers this many
// times fails with RAMBO_ENOMEM; before that it is requeued and retried.
constexpr uint32_t MAX_DEFERRALS = 64;
constexpr auto DEFER_BACKOFF = std::chrono::microseconds(200);

// Pinned host buffers for finished batches' large answers, reused across
// batches: a batch's IDs are copied from the device straight into one, its
// requests share it, and it returns to the pool when the last of them is
// collected.  Small answers go through the slot's pinned staging into heap
// memory instead, so uncollected small results hold no pinned memory.
struct PinnedPool {
    std::mutex mu;
    std::multimap<size_t, void*> free_bufs;  // capacity -> buffer
    std::vector<void*> all;
    ~PinnedPool() {
        for (void* p : all) cudaFreeHost(p);
    }
    void* get(size_t bytes, size_t* cap) {
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = free_bufs.lower_bound(bytes);
            if (it != free_bufs.end()) {
                void* p = it->second;
                *cap = it->first;
                free_bufs.erase(it);
                return p;
            }
        }
        size_t c = 1u << 20;
        while (c < bytes) c <<= 1;
        void* p = nullptr;
        if (cudaMallocHost(&p, c) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        std::lock_guard<std::mutex> lk(mu);
        all.push_back(p);
        *cap = c;
        return p;
    }
    void put(void* p, size_t cap) {
        std::lock_guard<std::mutex> lk(mu);
        free_bufs.emplace(cap, p);
    }
};

constexpr size_t SMALL_RESULT_BYTES = 256u << 10;

struct ResultBuf {
    std::shared_ptr<PinnedPool> pool;
    void* mem = nullptr;  // pooled pinned buffer (large answers)
    size_t cap = 0;
    std::vector<uint8_t> heap;  // small answers
    const uint32_t* ids = nullptr;
    ~ResultBuf() {
        if (mem) pool->put(mem, cap);
    }
};

struct Done {
    int status = 0;
    std::shared_ptr<const ResultBuf> buf;  // the batch's answers, shared by its requests
    uint64_t off = 0, len = 0;             // this request's run in buf
    uint64_t latency_ns = 0;
};

struct Slot {
    rambo_plan_t* plan = nullptr;
    cudaStream_t stream = nullptr;
    void* staging = nullptr;  // pinned, SMALL_RESULT_BYTES
    int kind = 1;
    bool busy = false;
    std::vector<Op> members;
};

}  // namespace

struct rambo_server {
    rambo_t* h = nullptr;
    rambo_server_config_t cfg{};
    int device = 0;
    std::vector<Slot> slots;
    cudaStream_t ins_stream = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Op> q[2];
    std::deque<Op> ins;
    std::unordered_map<uint64_t, Done> done;
    uint64_t next_ticket = 1, next_seq = 1, outstanding = 0;
    bool stop = false;
    std::thread worker;
    std::shared_ptr<PinnedPool> pool = std::make_shared<PinnedPool>();
    // pinned-memory refusals: injected ones (host-side test hook), deferral
    // count, and the time before which no new batch is admitted
    std::atomic<uint32_t> inject_alloc_fail{0};
    uint64_t n_deferred = 0;
    Clock::time_point backoff_until{};
    // statistics
    uint64_t n_queries = 0, n_batches = 0, n_inserts = 0, keys_done = 0;
    std::atomic<uint64_t> admit_ns{0}, finish_ns{0}, insert_ns{0}, idle_ns{0};
    std::vector<uint64_t> latencies;
    Clock::time_point t_first{}, t_last{};
    bool any = false;
};

namespace {

uint64_t op_keys(const Op& op) {
    if (op.kind == 0) return op.items;
    const uint32_t k = op.k & 0xffu;
    return op.items >= k ? op.items - k + 1 : 0;
}

uint64_t ns_since(Clock::time_point t0) {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
}

void finish_slot(rambo_server* S, Slot& sl) {
    const auto t0 = Clock::now();
    const uint32_t* d_ids = nullptr;
    const uint64_t* d_off = nullptr;
    uint64_t n_ids = 0;
    int rc = rambo_plan_wait(sl.plan, 0, &d_ids, &d_off, &n_ids, sl.stream);
    // the batch's offsets and IDs go from the device into one pooled pinned
    // buffer, which the batch's requests share
    const uint64_t nq = sl.members.size();
    std::shared_ptr<ResultBuf> buf;
    const uint64_t* off = nullptr;
    bool refused = false;  // no pinned memory for the answers
    if (rc == RAMBO_OK) {
        buf = std::make_shared<ResultBuf>();
        buf->pool = S->pool;
        const size_t off_bytes = (nq + 1) * 8, bytes = off_bytes + n_ids * 4;
        const bool small = bytes <= SMALL_RESULT_BYTES;
        void* dst = sl.staging;
        if (!small) {
            // a refusal injected by rambo_server_inject_alloc_failures stands in for cudaMallocHost failing
            uint32_t inj = S->inject_alloc_fail.load();
            while (inj && !S->inject_alloc_fail.compare_exchange_weak(inj, inj - 1)) {
            }
            dst = inj ? nullptr : (buf->mem = S->pool->get(bytes, &buf->cap));
        }
        if (!dst) {
            rc = RAMBO_ENOMEM;
            refused = true;
        } else {
            uint8_t* base = static_cast<uint8_t*>(dst);
            bool ok = cudaMemcpyAsync(base, d_off, off_bytes, cudaMemcpyDeviceToHost, sl.stream) == cudaSuccess;
            if (ok && n_ids)
                ok = cudaMemcpyAsync(base + off_bytes, d_ids, n_ids * 4, cudaMemcpyDeviceToHost, sl.stream) ==
                     cudaSuccess;
            ok = ok && cudaStreamSynchronize(sl.stream) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                rc = RAMBO_ECUDA;
            } else if (small) {
                buf->heap.assign(base, base + bytes);
                base = buf->heap.data();
            }
            off = reinterpret_cast<const uint64_t*>(base);
            buf->ids = reinterpret_cast<const uint32_t*>(base + off_bytes);
        }
    }
    const auto now = Clock::now();
    if (refused) {
        // no pinned memory for the answers: defer the batch -- its queries go
        // back to the front of the queue and run again after a short
        // back-off (collected results return buffers to the pool meanwhile);
        // a query deferred MAX_DEFERRALS times fails with RAMBO_ENOMEM
        std::lock_guard<std::mutex> lk(S->mu);
        auto& qq = S->q[sl.kind];
        for (auto it = sl.members.rbegin(); it != sl.members.rend(); ++it) {
            if (++it->deferrals <= MAX_DEFERRALS) {
                qq.push_front(std::move(*it));
                ++S->n_deferred;
                continue;
            }
            Done d;
            d.status = RAMBO_ENOMEM;
            d.latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - it->t_submit).count();
            S->done.emplace(it->ticket, std::move(d));
            --S->outstanding;
        }
        sl.members.clear();
        sl.busy = false;
        S->backoff_until = now + DEFER_BACKOFF;
        S->cv_work.notify_one();
        S->cv_done.notify_all();
        S->finish_ns += ns_since(t0);
        return;
    }
    if (rc == RAMBO_ENOSPC && sl.members.size() > 1) {
        // the batch's answers did not fit the slot: requeue its queries at the
        // front, each to run alone (their order among queries does not matter)
        std::lock_guard<std::mutex> lk(S->mu);
        auto& qq = S->q[sl.kind];
        for (auto it = sl.members.rbegin(); it != sl.members.rend(); ++it) {
            it->solo = true;
            qq.push_front(std::move(*it));
        }
        sl.members.clear();
        sl.busy = false;
        S->cv_work.notify_one();
        S->finish_ns += ns_since(t0);
        return;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (size_t i = 0; i < sl.members.size(); ++i) {
            const Op& op = sl.members[i];
            Done d;
            // a query whose own answer overflows the slot cannot be served:
            // RAMBO_E2BIG (RAMBO_ENOSPC from rambo_server_result means only
            // that the caller's buffer is too small)
            d.status = rc == RAMBO_ENOSPC ? RAMBO_E2BIG : rc;
            if (rc == RAMBO_OK) {
                d.buf = buf;
                d.off = off[i];
                d.len = off[i + 1] - off[i];
            }
            d.latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - op.t_submit).count();
            S->latencies.push_back(d.latency_ns);
            S->keys_done += op_keys(op);
            S->done.emplace(op.ticket, std::move(d));
            --S->outstanding;
        }
        S->n_queries += sl.members.size();
        S->n_batches += 1;
        S->t_last = now;
    }
    sl.members.clear();
    sl.busy = false;
    S->cv_done.notify_all();
    S->finish_ns += ns_since(t0);
}

// Takes queued queries of the slot's kind that precede every pending insert
// and fit the plan; caller holds the lock.
bool admit(rambo_server* S, Slot& sl) {
    auto& qq = S->q[sl.kind];
    const uint64_t barrier = S->ins.empty() ? ~0ull : S->ins.front().seq;
    const uint64_t max_q = sl.kind == 0 ? S->cfg.max_batch_queries : S->cfg.max_batch_queries;
    const uint64_t max_items = sl.kind == 0 ? S->cfg.max_batch_keys : S->cfg.max_batch_bases;
    uint64_t n = 0, items = 0;
    while (!qq.empty() && qq.front().seq < barrier && n < max_q && items + qq.front().items <= max_items) {
        if (qq.front().solo && n > 0) break;  // a requeued query rides alone
        const bool solo = qq.front().solo;
        items += qq.front().items;
        sl.members.push_back(std::move(qq.front()));
        qq.pop_front();
        ++n;
        if (solo) break;
    }
    if (!n) return false;
    void* hd = nullptr;
    uint64_t* ho = nullptr;
    rambo_plan_buffers(sl.plan, &hd, &ho, nullptr, nullptr);
    uint8_t* dst = static_cast<uint8_t*>(hd);
    const size_t elem = sl.kind == 0 ? 8 : 1;
    uint64_t at = 0;
    ho[0] = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const Op& op = sl.members[i];
        std::memcpy(dst + at * elem, op.data.data(), op.items * elem);
        at += op.items;
        ho[i + 1] = at;
    }
    const int rc = rambo_plan_launch(sl.plan, n, items, 1, sl.stream);
    if (rc) {
        // complete the batch with the launch error
        const auto now = Clock::now();
        for (auto& op : sl.members) {
            Done d;
            d.status = rc;
            d.latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - op.t_submit).count();
            S->done.emplace(op.ticket, std::move(d));
            --S->outstanding;
        }
        sl.members.clear();
        S->cv_done.notify_all();
        return false;
    }
    sl.busy = true;
    if (!S->any) {
        S->any = true;
        S->t_first = Clock::now();
    }
    return true;
}

void worker_main(rambo_server* S) {
    cudaSetDevice(S->device);
    const auto idle = std::chrono::microseconds(S->cfg.idle_wait_us ? S->cfg.idle_wait_us : 20);
    for (;;) {
        bool did = false;
        for (auto& sl : S->slots)
            if (sl.busy && rambo_plan_poll(sl.plan) != 1) {
                finish_slot(S, sl);
                did = true;
            }
        std::unique_lock<std::mutex> lk(S->mu);
        bool any_busy = false;
        for (auto& sl : S->slots) any_busy |= sl.busy;
        if (S->stop && S->q[0].empty() && S->q[1].empty() && S->ins.empty() && !any_busy) break;
        // an insert runs once everything submitted before it has finished
        if (!S->ins.empty() && !any_busy) {
            const uint64_t bseq = S->ins.front().seq;
            const bool earlier_q = (!S->q[0].empty() && S->q[0].front().seq < bseq) ||
                                   (!S->q[1].empty() && S->q[1].front().seq < bseq);
            if (!earlier_q) {
                Op op = std::move(S->ins.front());
                S->ins.pop_front();
                lk.unlock();
                const auto t_ins = Clock::now();
                int rc;
                if (op.kind == 0)
                    rc = rambo_insert_batch(S->h, op.set_ids.data(), reinterpret_cast<const uint64_t*>(op.data.data()),
                                            op.offsets.data(), op.set_ids.size(), 0, S->ins_stream);
                else
                    rc = rambo_insert_seq_batch(S->h, op.set_ids.data(), op.data.data(), op.offsets.data(),
                                                op.set_ids.size(), op.k, 0, S->ins_stream);
                S->insert_ns += ns_since(t_ins);
                lk.lock();
                Done d;
                d.status = rc;
                d.latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() -
                                                                                              op.t_submit)
                                   .count();
                S->done.emplace(op.ticket, std::move(d));
                --S->outstanding;
                ++S->n_inserts;
                S->cv_done.notify_all();
                did = true;
            }
        }
        const auto t_adm = Clock::now();
        bool launched = false;
        if (t_adm >= S->backoff_until)  // (after a pinned-memory refusal, admission pauses briefly)
            for (auto& sl : S->slots)
                if (!sl.busy && admit(S, sl)) launched = true;
        if (launched) S->admit_ns += ns_since(t_adm);
        did |= launched;
        if (!did) {
            const auto t_idle = Clock::now();
            S->cv_work.wait_for(lk, idle);
            S->idle_ns += ns_since(t_idle);
        }
    }
}

int submit_op(rambo_server* S, Op&& op, uint64_t* ticket) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return RAMBO_ESTATE;
    op.ticket = S->next_ticket++;
    op.seq = S->next_seq++;
    op.t_submit = Clock::now();
    if (ticket) *ticket = op.ticket;
    ++S->outstanding;
    if (op.type == 1) S->ins.push_back(std::move(op));
    else S->q[op.kind].push_back(std::move(op));
    S->cv_work.notify_one();
    return RAMBO_OK;
}

}  // namespace

extern "C" {

int rambo_server_create(rambo_t* h, const rambo_server_config_t* cfg, rambo_server_t** out) {
    if (!h || !cfg || !out || cfg->slots < 1 || cfg->slots > 16 || !cfg->max_batch_queries || !cfg->max_batch_ids ||
        (!cfg->max_batch_bases && !cfg->max_batch_keys))
        return RAMBO_EINVAL;
    {
        uint32_t kk = 0;
        int canon = 0;
        if (!rgb::split_k(cfg->k, &kk, &canon)) return RAMBO_EINVAL;
    }
    *out = nullptr;
    rambo_server* S = new (std::nothrow) rambo_server();
    if (!S) return RAMBO_ENOMEM;
    S->h = h;
    S->cfg = *cfg;
    cudaGetDevice(&S->device);
    int rc = RAMBO_OK;
    for (int kind = 0; kind < 2 && rc == RAMBO_OK; ++kind) {
        const uint64_t items = kind == 0 ? cfg->max_batch_keys : cfg->max_batch_bases;
        if (!items) continue;
        for (uint32_t i = 0; i < cfg->slots && rc == RAMBO_OK; ++i) {
            Slot sl;
            sl.kind = kind;
            rc = rambo_plan_create(h, kind, cfg->max_batch_queries, items, cfg->max_batch_ids, cfg->k, &sl.plan);
            // replays without timing nodes: the server reports latency, not kernel times
            if (rc == RAMBO_OK) rambo_plan_set_timing(sl.plan, 0);
            if (rc == RAMBO_OK && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess)
                rc = RAMBO_ECUDA;
            if (rc == RAMBO_OK && cudaMallocHost(&sl.staging, SMALL_RESULT_BYTES) != cudaSuccess) {
                cudaGetLastError();
                rc = RAMBO_ENOMEM;
            }
            S->slots.push_back(sl);
        }
    }
    if (rc == RAMBO_OK && cudaStreamCreateWithFlags(&S->ins_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = RAMBO_ECUDA;
    if (rc != RAMBO_OK) {
        for (auto& sl : S->slots) {
            if (sl.plan) rambo_plan_destroy(sl.plan);
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.staging) cudaFreeHost(sl.staging);
        }
        if (S->ins_stream) cudaStreamDestroy(S->ins_stream);
        delete S;
        return rc;
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return RAMBO_OK;
}

int rambo_server_submit(rambo_server_t* S, int kind, const void* data, uint64_t n_items, uint64_t* ticket) {
    if (!S || (kind != 0 && kind != 1) || (!data && n_items)) return RAMBO_EINVAL;
    const uint64_t cap = kind == 0 ? S->cfg.max_batch_keys : S->cfg.max_batch_bases;
    if (n_items > cap) return RAMBO_E2BIG;  // larger than a whole slot: cannot be admitted
    Op op;
    op.type = 0;
    op.kind = kind;
    op.items = n_items;
    op.k = S->cfg.k;
    const size_t bytes = n_items * (kind == 0 ? 8 : 1);
    op.data.assign(static_cast<const uint8_t*>(data), static_cast<const uint8_t*>(data) + bytes);
    return submit_op(S, std::move(op), ticket);
}

int rambo_server_submit_insert(rambo_server_t* S, int kind, const uint64_t* set_ids, const void* data,
                               const uint64_t* offsets, uint64_t n_sets, uint64_t* ticket) {
    if (!S || (kind != 0 && kind != 1) || !offsets || (!set_ids && n_sets)) return RAMBO_EINVAL;
    if (offsets[n_sets] < offsets[0]) return RAMBO_EINVAL;
    Op op;
    op.type = 1;
    op.kind = kind;
    op.k = S->cfg.k;
    op.set_ids.assign(set_ids, set_ids + n_sets);
    op.offsets.resize(n_sets + 1);
    for (uint64_t t = 0; t <= n_sets; ++t) op.offsets[t] = offsets[t] - offsets[0];
    const size_t elem = kind == 0 ? 8 : 1;
    const uint8_t* d = static_cast<const uint8_t*>(data) + offsets[0] * elem;
    op.data.assign(d, d + (offsets[n_sets] - offsets[0]) * elem);
    op.items = offsets[n_sets] - offsets[0];
    return submit_op(S, std::move(op), ticket);
}

int rambo_server_result(rambo_server_t* S, uint64_t ticket, int wait, uint32_t* ids, uint64_t cap, uint64_t* n_ids,
                        uint64_t* latency_ns) {
    if (!S) return RAMBO_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    while (it == S->done.end()) {
        if (!wait) return 1;
        S->cv_done.wait(lk);
        it = S->done.find(ticket);
    }
    Done& d = it->second;
    if (n_ids) *n_ids = d.len;
    if (latency_ns) *latency_ns = d.latency_ns;
    if (d.status != RAMBO_OK) {
        const int rc = d.status;
        S->done.erase(it);
        return rc;
    }
    if (d.len > cap) return RAMBO_ENOSPC;  // kept: ask again with a larger buffer
    // take the request's share of the batch buffer, then copy without the lock
    const std::shared_ptr<const ResultBuf> buf = d.buf;
    const uint64_t off = d.off, len = d.len;
    S->done.erase(it);
    lk.unlock();
    if (len) std::memcpy(ids, buf->ids + off, len * 4);
    return RAMBO_OK;
}

int rambo_server_drain(rambo_server_t* S) {
    if (!S) return RAMBO_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_work.notify_one();
    while (S->outstanding) S->cv_done.wait(lk);
    return RAMBO_OK;
}

int rambo_server_stats(rambo_server_t* S, rambo_server_stats_t* out) {
    if (!S || !out) return RAMBO_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->queries = S->n_queries;
    out->batches = S->n_batches;
    out->inserts = S->n_inserts;
    out->keys = S->keys_done;
    out->seconds = S->any ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
    out->admit_ns = S->admit_ns;
    out->finish_ns = S->finish_ns;
    out->insert_ns = S->insert_ns;
    out->idle_ns = S->idle_ns;
    out->deferred = S->n_deferred;
    if (!S->latencies.empty()) {
        std::vector<uint64_t> l = S->latencies;
        std::sort(l.begin(), l.end());
        out->p50_ns = l[l.size() / 2];
        out->p99_ns = l[std::min(l.size() - 1, (size_t)(0.99 * (double)l.size()))];
        out->max_ns = l.back();
    }
    return RAMBO_OK;
}

int rambo_server_reset_stats(rambo_server_t* S) {
    if (!S) return RAMBO_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    S->n_queries = S->n_batches = S->n_inserts = S->keys_done = 0;
    S->admit_ns = S->finish_ns = S->insert_ns = S->idle_ns = 0;
    S->n_deferred = 0;
    S->latencies.clear();
    S->any = false;
    return RAMBO_OK;
}

int rambo_server_inject_alloc_failures(rambo_server_t* S, uint32_t n) {
    if (!S) return RAMBO_EINVAL;
    S->inject_alloc_fail.store(n);
    return RAMBO_OK;
}

int rambo_server_replay(rambo_server_t* S, const uint8_t* kinds, const uint8_t* bytes, const uint64_t* byte_offsets,
                        const uint64_t* arrival_ns, uint64_t n, uint64_t* tickets) {
    if (!S || (!kinds && n) || !byte_offsets) return RAMBO_EINVAL;
    const auto t0 = Clock::now();
    for (uint64_t i = 0; i < n; ++i) {
        const auto when = t0 + std::chrono::nanoseconds(arrival_ns ? arrival_ns[i] : 0);
        while (Clock::now() < when) {
            const auto left = when - Clock::now();
            if (left > std::chrono::microseconds(200)) std::this_thread::sleep_for(left - std::chrono::microseconds(100));
        }
        const int kind = kinds[i];
        const uint64_t nb = byte_offsets[i + 1] - byte_offsets[i];
        const uint64_t items = kind == 0 ? nb / 8 : nb;
        const int rc = rambo_server_submit(S, kind, bytes + byte_offsets[i], items, tickets ? tickets + i : nullptr);
        if (rc) return rc;
    }
    return RAMBO_OK;
}

void rambo_server_destroy(rambo_server_t* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto& sl : S->slots) {
        if (sl.plan) rambo_plan_destroy(sl.plan);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.staging) cudaFreeHost(sl.staging);
    }
    if (S->ins_stream) cudaStreamDestroy(S->ins_stream);
    delete S;
}

}  // extern "C"
