// rambo_plan.cu -- graph-captured query plans.
//
// A plan owns device buffers sized for a maximum batch (queries, bases or
// keys, result IDs) and a CUDA graph captured once at creation: descriptor
// upload, status reset, validation, 2-bit packing, the persistent query
// kernel, the count scan, the gather, and the copy of the status word back to
// pinned host memory.  Kernels read the batch size from the uploaded
// descriptor, so one captured graph replays for any batch up to capacity.
// A launch is asynchronous; the host learns the result size from the status
// copy and then copies exactly the IDs it needs.  Each plan has its own
// status block and buffers, so several plans run concurrently on different
// streams against the same (read-only) index.
#include <cstring>
#include <new>

#include "k_query.cuh"
#include "rambo_impl.cuh"

using namespace rgb;

namespace {

int map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return RAMBO_OK;
    return e == cudaErrorMemoryAllocation ? RAMBO_ENOMEM : RAMBO_ECUDA;
}

#define PK(x)                                      \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) return map_cuda(e_); \
    } while (0)

// What one host-to-device copy node writes before every replay: the batch
// descriptor {n, total} and a clean status block (error words, work-queue
// ticket, cursor, counters), so no reset kernel is needed.
struct PlanHead {
    uint64_t desc[2];
    uint64_t pad[2];
    DevStatus st;
};

}  // namespace

struct rambo_plan {
    rambo_t* h = nullptr;
    int kind = 1;
    uint32_t k = 31;
    int canon = 0, skipn = 0;
    uint64_t max_q = 0, max_items = 0, max_ids = 0;
    uint64_t stage_words = 0;  // staging arena: max_ids, or less when dense answers are staged as bitmaps
    uint32_t staging = 0;      // answer staging form at creation (see set_staging)
    int device = 0;
    size_t elem = 1;
    // device
    uint8_t* d_data = nullptr;
    uint64_t* d_off = nullptr;
    uint64_t* d_packed = nullptr;
    uint32_t* d_nmask = nullptr;  // skip-N: unresolved-base bits
    uint32_t* qcount = nullptr;
    uint64_t* qstart = nullptr;
    uint64_t* scan_tmp = nullptr;
    uint32_t* stage = nullptr;
    uint32_t* ids = nullptr;
    uint64_t* id_off = nullptr;
    PlanHead* d_head = nullptr;
    DevStatus* st = nullptr;   // &d_head->st
    uint64_t* d_desc = nullptr;  // d_head->desc
    // pinned host
    uint8_t* h_data = nullptr;
    uint64_t* h_off = nullptr;
    PlanHead* h_head = nullptr;  // descriptor + clean status template
    uint64_t* h_desc = nullptr;  // h_head->desc
    DevStatus* h_st = nullptr;
    uint32_t* h_ids = nullptr;
    uint64_t* h_id_off = nullptr;
    // graph
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;        // with the timing nodes (null if they could not be captured)
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph_plain = nullptr;  // the same work without them
    cudaGraphExec_t exec_plain = nullptr;
    bool use_timed = true;              // rambo_plan_set_timing
    cudaEvent_t ev_done = nullptr;
    // timing events recorded by nodes of the graph itself: replay start,
    // query kernel start and end, replay end (null when not captured)
    cudaEvent_t ev_t[4] = {nullptr, nullptr, nullptr, nullptr};
    bool timed = false;
    rambo_query_stats_t last{};
    uint64_t launched_n = 0;
    bool busy = false;
    bool attached = false;  // counted in the handle's live plans
    int launches_per_replay = 0;
};

namespace {

void plan_free(rambo_plan* p) {
    if (!p) return;
    if (p->attached && p->h) handle_detach_plan(p->h, p);
    cudaSetDevice(p->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->exec_plain) cudaGraphExecDestroy(p->exec_plain);
    if (p->graph_plain) cudaGraphDestroy(p->graph_plain);
    if (p->ev_done) cudaEventDestroy(p->ev_done);
    for (cudaEvent_t e : p->ev_t)
        if (e) cudaEventDestroy(e);
    if (p->cap) cudaStreamDestroy(p->cap);
    void* dev[] = {p->d_data, p->d_off, p->d_packed, p->d_nmask, p->qcount, p->qstart, p->scan_tmp,
                   p->stage, p->ids, p->id_off, p->d_head};
    for (void* d : dev)
        if (d) cudaFree(d);
    void* host[] = {p->h_data, p->h_off, p->h_head, p->h_st, p->h_ids, p->h_id_off};
    for (void* x : host)
        if (x) cudaFreeHost(x);
    delete p;
}

// Records timing event i inside the captured graph (an event-record node).
cudaError_t mark(rambo_plan* p, int i, cudaStream_t s, bool timed) {
    return timed ? cudaEventRecordWithFlags(p->ev_t[i], s, cudaEventRecordExternal) : cudaSuccess;
}

int plan_capture(rambo_plan* p, bool timed) {
    IndexView ix;
    HashParams hp;
    QueryTuning t;
    int use_bitmap = 0, dev = 0;
    int rc = handle_query_view(p->h, p->max_q, &ix, &hp, &t, &use_bitmap, &dev);
    if (rc) return rc;
    BatchView b{};
    b.seq = p->kind;
    b.offsets = p->d_off;
    b.keys = p->kind == 0 ? reinterpret_cast<const uint64_t*>(p->d_data) : nullptr;
    b.packed = p->kind == 1 ? p->d_packed : nullptr;
    b.n = p->max_q;
    b.total = p->max_items;
    b.off0 = 0;
    b.k = p->k;
    b.canon = p->canon;
    b.skipn = p->skipn;
    b.nmask = p->d_nmask;
    b.desc = p->d_desc;
    const uint64_t scan_words = scan_tmp_words(p->max_q);
    cudaStream_t s = p->cap;
    PK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = mark(p, 0, s, timed);
    // descriptor and clean status block in one copy node
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_head, p->h_head, sizeof(PlanHead), cudaMemcpyHostToDevice, s);
    int n_launch = 0;
    // intake: validation and (DNA) packing in one kernel
    if (e == cudaSuccess)
        e = launch_intake(b, p->kind ? p->k : 1, ix.K, p->kind == 1 ? p->d_data : nullptr, p->d_packed,
                          p->kind == 1 ? p->max_items / 32 + 2 : 0, p->d_nmask, p->st, s),
        ++n_launch;
    if (e == cudaSuccess && p->kind == 1 && p->skipn) e = launch_check_windows(b, p->st, s), ++n_launch;
    QueryOut o{p->stage, p->stage_words, p->qstart, p->qcount, 0, 0};
    set_staging(o, ix.K, p->staging);
    if (e == cudaSuccess) e = mark(p, 1, s, timed);
    if (e == cudaSuccess) {
        int nq = 0;
        e = launch_query(ix, hp, b, o, t, use_bitmap, p->st, s, &nq);
        n_launch += nq;
    }
    if (e == cudaSuccess) e = mark(p, 2, s, timed);
    if (e == cudaSuccess) {
        int n_scan = 0;
        // the scan also stores the number of result IDs in the status block
        e = launch_scan_counts(p->qcount, p->max_q, p->id_off, p->scan_tmp, scan_words, s, p->d_desc, &n_scan,
                               nullptr, &p->st->spare[1]);
        n_launch += n_scan;
    }
    if (e == cudaSuccess) e = launch_gather(o, p->id_off, p->max_q, p->ids, p->st, s, p->d_desc, p->max_ids);
    ++n_launch;
    if (e == cudaSuccess) e = mark(p, 3, s, timed);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->h_st, p->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return map_cuda(e != cudaSuccess ? e : e2);
    }
    cudaGraph_t& graph = timed ? p->graph : p->graph_plain;
    cudaGraphExec_t& exec = timed ? p->exec : p->exec_plain;
    graph = g;
    PK(cudaGraphInstantiate(&exec, g, 0));
    p->launches_per_replay = n_launch;
    return RAMBO_OK;
}

int decode(unsigned long long e) {
    if (e == NO_ERR) return RAMBO_OK;
    switch ((unsigned)(e & 0xff)) {
        case PRIO_ERANGE: return RAMBO_ERANGE;
        case PRIO_EINVAL: return RAMBO_EINVAL;
        case PRIO_EBADSEQ: return RAMBO_EBADSEQ;
        default: return RAMBO_ECUDA;
    }
}

}  // namespace

namespace rgb {
// The plan's handle is being destroyed: its captured graph now points to freed
// memory, so the plan forgets the handle and refuses further launches.
void plan_orphan(rambo_plan_t* p) {
    if (!p) return;
    if (p->busy) cudaEventSynchronize(p->ev_done);
    p->busy = false;
    p->h = nullptr;
    p->attached = false;
}
}  // namespace rgb

extern "C" {

int rambo_plan_create(rambo_t* h, int kind, uint64_t max_queries, uint64_t max_items, uint64_t max_ids, uint32_t k,
                      rambo_plan_t** out) {
    if (!h || !out || (kind != 0 && kind != 1) || !max_queries || !max_items || !max_ids) return RAMBO_EINVAL;
    uint32_t kk = 0;
    int canon = 0, skipn = 0;
    if (kind == 1 && !split_k(k, &kk, &canon, &skipn)) return RAMBO_EINVAL;
    if (max_queries > 0xffffffffull) return RAMBO_EINVAL;
    *out = nullptr;
    rambo_plan* p = new (std::nothrow) rambo_plan();
    if (!p) return RAMBO_ENOMEM;
    IndexView ix;
    HashParams hp;
    QueryTuning t;
    int ub = 0;
    int rc = handle_query_view(h, max_queries, &ix, &hp, &t, &ub, &p->device);
    if (rc) {
        delete p;
        return rc;
    }
    p->h = h;
    p->kind = kind;
    p->k = kind == 1 ? kk : 0;
    p->canon = kind == 1 ? canon : 0;
    p->skipn = kind == 1 ? skipn : 0;
    p->max_q = max_queries;
    p->max_items = max_items;
    p->max_ids = max_ids;
    // a query stages at most ceil(K/32) words when the kernel keeps its set
    // bitmap (denser answers are staged as the bitmap), never more than its IDs
    p->stage_words = max_ids;
    p->staging = t.staging;
    if (ub && !t.wide) {
        QueryOut form{};
        set_staging(form, ix.K, t.staging);
        if (form.bits_words && max_queries <= max_ids / form.bits_min) p->stage_words = max_queries * form.bits_min;
    }
    p->elem = kind == 0 ? 8 : 1;
    auto fail = [&](int code) {
        plan_free(p);
        return code;
    };
    if (cudaSetDevice(p->device) != cudaSuccess) return fail(RAMBO_ECUDA);
    bool ok = cudaMalloc(&p->d_data, max_items * p->elem + 16) == cudaSuccess &&
              cudaMalloc(&p->d_off, (max_queries + 1) * 8) == cudaSuccess &&
              (kind == 0 || cudaMalloc(&p->d_packed, (max_items / 32 + 2) * 8) == cudaSuccess) &&
              (!p->skipn || cudaMalloc(&p->d_nmask, (max_items / 32 + 2) * 4) == cudaSuccess) &&
              cudaMalloc(&p->qcount, max_queries * 4) == cudaSuccess &&
              cudaMalloc(&p->qstart, max_queries * 8) == cudaSuccess &&
              cudaMalloc(&p->scan_tmp, scan_tmp_words(max_queries) * 8) == cudaSuccess &&
              cudaMalloc(&p->stage, p->stage_words * 4) == cudaSuccess && cudaMalloc(&p->ids, max_ids * 4) == cudaSuccess &&
              cudaMalloc(&p->id_off, (max_queries + 1) * 8) == cudaSuccess &&
              cudaMalloc(&p->d_head, sizeof(PlanHead)) == cudaSuccess &&
              cudaMallocHost(&p->h_data, max_items * p->elem + 16) == cudaSuccess &&
              cudaMallocHost(&p->h_off, (max_queries + 1) * 8) == cudaSuccess &&
              cudaMallocHost(&p->h_head, sizeof(PlanHead)) == cudaSuccess &&
              cudaMallocHost(&p->h_st, sizeof(DevStatus)) == cudaSuccess &&
              cudaMallocHost(&p->h_ids, max_ids * 4) == cudaSuccess &&
              cudaMallocHost(&p->h_id_off, (max_queries + 1) * 8) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return fail(RAMBO_ENOMEM);
    }
    p->st = &p->d_head->st;
    p->d_desc = p->d_head->desc;
    p->h_desc = p->h_head->desc;
    *p->h_head = PlanHead{};
    p->h_head->st.err = NO_ERR;
    p->h_head->st.bad_pos = NO_ERR;
    if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_done, cudaEventDisableTiming) != cudaSuccess)
        return fail(RAMBO_ECUDA);
    for (cudaEvent_t& ev : p->ev_t)
        if (cudaEventCreate(&ev) != cudaSuccess) return fail(RAMBO_ECUDA);
    p->h_desc[0] = 0;
    p->h_desc[1] = 0;
    // the graph without timing nodes, then the one with them (the default
    // when it can be captured; both answer the same)
    rc = plan_capture(p, false);
    if (rc) return fail(rc);
    if (plan_capture(p, true) != RAMBO_OK) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        p->exec = nullptr;
        p->graph = nullptr;
        cudaGetLastError();
    }
    handle_attach_plan(h, p);
    p->attached = true;
    *out = p;
    return RAMBO_OK;
}

void rambo_plan_destroy(rambo_plan_t* p) {
    if (p && p->busy) cudaEventSynchronize(p->ev_done);
    plan_free(p);
}

int rambo_plan_buffers(rambo_plan_t* p, void** host_data, uint64_t** host_offsets, void** dev_data,
                       uint64_t** dev_offsets) {
    if (!p) return RAMBO_EINVAL;
    if (host_data) *host_data = p->h_data;
    if (host_offsets) *host_offsets = p->h_off;
    if (dev_data) *dev_data = p->d_data;
    if (dev_offsets) *dev_offsets = p->d_off;
    return RAMBO_OK;
}

int rambo_plan_launch(rambo_plan_t* p, uint64_t n_queries, uint64_t n_items, int from_host, void* stream) {
    if (!p || n_queries == 0) return RAMBO_EINVAL;
    if (p->busy || !p->h) return RAMBO_ESTATE;  // running, or its handle was destroyed
    if (n_queries > p->max_q || n_items > p->max_items) return RAMBO_E2BIG;
    cudaStream_t s = (cudaStream_t)stream;
    PK(cudaSetDevice(p->device));
    p->h_desc[0] = n_queries;
    p->h_desc[1] = n_items;
    if (from_host) {
        PK(cudaMemcpyAsync(p->d_off, p->h_off, (n_queries + 1) * 8, cudaMemcpyHostToDevice, s));
        if (n_items) PK(cudaMemcpyAsync(p->d_data, p->h_data, n_items * p->elem, cudaMemcpyHostToDevice, s));
    }
    p->timed = p->use_timed && p->exec;
    PK(cudaGraphLaunch(p->timed ? p->exec : p->exec_plain, s));
    PK(cudaEventRecord(p->ev_done, s));
    p->launched_n = n_queries;
    p->busy = true;
    return RAMBO_OK;
}

int rambo_plan_poll(rambo_plan_t* p) {
    if (!p) return RAMBO_EINVAL;
    if (!p->busy) return RAMBO_ESTATE;
    cudaError_t e = cudaEventQuery(p->ev_done);
    if (e == cudaErrorNotReady) return 1;
    return map_cuda(e);
}

int rambo_plan_wait(rambo_plan_t* p, int to_host, const uint32_t** ids, const uint64_t** id_offsets, uint64_t* n_ids,
                    void* stream) {
    if (!p) return RAMBO_EINVAL;
    if (!p->busy) return RAMBO_ESTATE;
    PK(cudaSetDevice(p->device));
    PK(cudaEventSynchronize(p->ev_done));
    p->busy = false;
    const DevStatus st = *p->h_st;
    int rc = decode(st.err);
    if (rc) return rc;
    const uint64_t total = st.spare[1];
    p->last = rambo_query_stats_t{};
    p->last.n_queries = p->launched_n;
    p->last.keys_submitted = p->kind == 1 ? p->h_desc[1] - p->launched_n * (uint64_t)(p->k - 1) : p->h_desc[1];
    p->last.keys_probed = st.keys_probed;
    p->last.rows_read = st.rows_read;
    p->last.n_results = total;
    p->last.kernel_launches = (uint64_t)p->launches_per_replay;
    for (int i = 0; i < 4; ++i) p->last.stage_queries[i] = st.stage_count[i];
    p->last.staged_words = st.cursor;
    if (p->timed) {
        PK(cudaEventElapsedTime(&p->last.query_kernel_ms, p->ev_t[1], p->ev_t[2]));
        PK(cudaEventElapsedTime(&p->last.device_ms, p->ev_t[0], p->ev_t[3]));
    }
    if (n_ids) *n_ids = total;
    if (st.cursor > p->stage_words || total > p->max_ids) return RAMBO_ENOSPC;
    const uint64_t n = p->launched_n;
    if (to_host) {
        cudaStream_t s = (cudaStream_t)stream;
        PK(cudaMemcpyAsync(p->h_id_off, p->id_off, (n + 1) * 8, cudaMemcpyDeviceToHost, s));
        if (total) PK(cudaMemcpyAsync(p->h_ids, p->ids, total * 4, cudaMemcpyDeviceToHost, s));
        PK(cudaStreamSynchronize(s));
        if (ids) *ids = p->h_ids;
        if (id_offsets) *id_offsets = p->h_id_off;
    } else {
        if (ids) *ids = p->ids;
        if (id_offsets) *id_offsets = p->id_off;
    }
    return RAMBO_OK;
}

int rambo_plan_launches_per_replay(const rambo_plan_t* p) { return p ? p->launches_per_replay : 0; }

int rambo_plan_set_timing(rambo_plan_t* p, int on) {
    if (!p || (on != 0 && on != 1)) return RAMBO_EINVAL;
    if (p->busy) return RAMBO_ESTATE;
    if (on && !p->exec) return RAMBO_ECUDA;  // the timed graph could not be captured
    p->use_timed = on != 0;
    return RAMBO_OK;
}

int rambo_plan_last_stats(const rambo_plan_t* p, rambo_query_stats_t* out) {
    if (!p || !out) return RAMBO_EINVAL;
    *out = p->last;
    return RAMBO_OK;
}

}  // extern "C"
