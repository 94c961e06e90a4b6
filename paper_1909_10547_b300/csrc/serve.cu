// Continuously batched serving of FK convolutions over device-resident
// tables (the paper's point that the accelerator pays off once the transfer
// penalty is overcome, Sec. 3: tables stay on the device, only PDFs and
// observables move, and many requests share the device at once).
//
// One scheduler thread per server:
//  - admission: FIFO; a request is admitted while fewer than max_inflight
//    batches run and the device bytes of the admitted work plus the resident
//    tables stay within the budget;
//  - coalescing: requests waiting on the same table and precision are joined
//    along the replica axis into one launch.  In FP64/FP32 the kernel (and so
//    the summation order of every observable) depends only on whether R <= 4,
//    so requests are joined only within that class and each result is bit
//    for bit the one the request would get alone; the tensor-core modes
//    compute every replica row independently of the others;
//  - each batch runs on its own stream: pinned H2D of the PDFs, the
//    convolution, D2H of each request's observables, then a host callback
//    marks the requests done and returns their bytes to the budget;
//  - failure detection: every failure ends in a per-ticket status.  A batch
//    whose completion callback has not arrived once its stream has finished
//    and a grace period has passed (a lost completion message) has its
//    requests failed with FK_ETIMEDOUT and its budget returned; a request can
//    be cancelled (FK_ECANCELED); destroying a server fails what never
//    started and waits for what is running.  Host-side faults (a failed
//    pinned or device allocation, a failed launch, a dropped completion) can
//    be injected with fk_serve_inject or the FK_FAULT environment variable,
//    to test these paths without any fault on the GPU.
#include "fk_internal.h"

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <string>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

namespace fk {
namespace {

struct Request;

struct Batch {
    struct fk_server *srv = nullptr;
    std::vector<Request *> reqs;
    size_t bytes = 0;
    int stream = 0;
    std::chrono::steady_clock::time_point t0;  // when its work was enqueued
};

// a batch whose completion message was lost, with an event after its work
struct Unconfirmed {
    Batch *b;
    cudaEvent_t ev;
};

struct Request {
    uint64_t ticket = 0;
    int table = 0, R = 0, prec = 0;
    size_t f_bytes = 0, o_bytes = 0, dev_bytes = 0;
    void *F = nullptr;  // pinned
    void *O = nullptr;  // pinned
    int status = FK_OK;
    bool done = false;
    bool cancelled = false;
};

// Pinned host buffers for request staging.  Pinning is slow (milliseconds per
// call), so memory is pinned in slabs of at least 64 MiB and carved into
// power-of-two size classes; freed buffers go back to their class's free list
// and are reused.  Everything is unpinned when the server is destroyed.
class PinnedPool {
   public:
    void *get(size_t n, size_t *cls) {
        size_t c = 4096;
        while (c < n) c <<= 1;
        *cls = c;
        std::lock_guard<std::mutex> l(mu_);
        auto &v = free_[c];
        if (!v.empty()) {
            void *p = v.back();
            v.pop_back();
            return p;
        }
        if (left_ < c) {
            const size_t slab = std::max<size_t>(c, SLAB);
            void *p = nullptr;
            if (cudaHostAlloc(&p, slab, cudaHostAllocDefault) != cudaSuccess) return nullptr;
            slabs_.push_back(p);
            cur_ = static_cast<char *>(p);
            left_ = slab;
        }
        void *p = cur_;
        cur_ += c;
        left_ -= c;
        return p;
    }
    void put(void *p, size_t cls) {
        if (!p) return;
        std::lock_guard<std::mutex> l(mu_);
        free_[cls].push_back(p);
    }
    ~PinnedPool() {
        for (void *p : slabs_) cudaFreeHost(p);
    }

   private:
    static constexpr size_t SLAB = 64u << 20;
    std::mutex mu_;
    std::map<size_t, std::vector<void *>> free_;
    std::vector<void *> slabs_;
    char *cur_ = nullptr;
    size_t left_ = 0;
};

size_t pow2_class(size_t n) {
    size_t c = 4096;
    while (c < n) c <<= 1;
    return c;
}

// Device bytes a launch of R replicas on table t needs besides the table.
size_t request_device_bytes(const fk_table *t, int R, int prec) {
    const size_t esz = FK_IO64(prec) ? 8 : 4;
    size_t b = esz * (size_t)R * NFL * t->nxg + esz * (size_t)R * t->ndata;
    if (prec == FK_FP64 || prec == FK_FP32) {
        b += esz * (size_t)R * t->ndata * 256;  // partial sums (the split is at most 196)
    } else if (prec == FK_FP64_TC) {
        // digit slices of the replicas' operand (8 x 2 bytes per element), the
        // PDF matrix (hadronic) and up to 1 GiB of exact partial tiles
        const size_t rpad = (size_t)(R + 127) / 128 * 128;
        b += rpad * t->tc.oz.ktot_pad * 16 + (t->kind == FK_KIND_HAD ? 8 * (size_t)R * t->E : 0) + (1ull << 30);
    } else if (t->tc.lum_on) {
        // the builders' transposed PDF rows and the partial tiles of the K splits
        const size_t rpad = (size_t)(R + 127) / 128 * 128;
        const size_t nsplit = (size_t)(t->tc.lum.ktot_pad + 1535) / 1536;
        b += 4 * rpad * NFL * t->nx + 4 * nsplit * R * t->ndata;
    } else {
        const size_t rpad = (size_t)(R + 127) / 128 * 128;
        b += rpad * t->tc.fwd.ktot_pad * (prec == FK_TF32 ? 4 : (prec == FK_BF16X3 ? 4 : 2)) +
             4 * rpad * (size_t)t->tc.fwd.grp.ngroups * t->nx;
    }
    return b + 4096;
}

}  // namespace
}  // namespace fk

using namespace fk;

struct fk_server {
    size_t budget = 0;
    int max_inflight = 1;
    int device = 0;
    std::vector<fk_table *> tables;
    size_t resident = 0;
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    PinnedPool pinned;

    std::mutex mu;
    std::condition_variable cv_sched;  // work or capacity changed
    std::condition_variable cv_done;   // a request finished
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    int inflight = 0;
    size_t inflight_bytes = 0;
    bool stop = false;
    std::thread worker;

    uint64_t completed = 0, dp_rep = 0, launches = 0;
    size_t peak_bytes = 0;

    // failure detection and injection
    int faults[FK_FAULT_DROP + 1] = {};   // armed host-side faults, by kind
    std::vector<Unconfirmed> unconfirmed; // batches whose completion message was lost
    int grace_ms = 200;                   // after the stream is idle, before a batch is given up
    uint64_t timed_out = 0;
};

namespace fk {
namespace {

// Takes one armed fault of this kind (caller holds s->mu or none is needed).
bool take_fault(fk_server *s, int kind) {
    std::lock_guard<std::mutex> l(s->mu);
    if (s->faults[kind] <= 0) return false;
    --s->faults[kind];
    return true;
}

// Batches whose completion message never came: once the work they enqueued
// has finished (their event) and the grace period has passed, their requests
// fail with FK_ETIMEDOUT and their budget is returned.  Caller holds s->mu.
bool reap_unconfirmed(fk_server *s) {
    auto &v = s->unconfirmed;
    bool any = false;
    const auto now = std::chrono::steady_clock::now();
    for (size_t i = 0; i < v.size();) {
        Batch *b = v[i].b;
        const bool finished = cudaEventQuery(v[i].ev) == cudaSuccess;
        if (finished && now - b->t0 > std::chrono::milliseconds(s->grace_ms)) {
            for (Request *r : b->reqs) {
                r->status = FK_ETIMEDOUT;
                r->done = true;
            }
            s->inflight--;
            s->inflight_bytes -= b->bytes;
            s->timed_out += b->reqs.size();
            cudaEventDestroy(v[i].ev);
            delete b;
            v.erase(v.begin() + i);
            any = true;
        } else {
            ++i;
        }
    }
    return any;
}

bool has_unconfirmed(const fk_server *s) { return !s->unconfirmed.empty(); }

void CUDART_CB batch_done(void *arg) {
    Batch *b = static_cast<Batch *>(arg);
    fk_server *s = b->srv;
    {
        std::lock_guard<std::mutex> l(s->mu);
        for (Request *r : b->reqs) {
            r->done = true;
            s->completed++;
            s->dp_rep += (uint64_t)r->R * s->tables[r->table]->ndata;
        }
        s->inflight--;
        s->inflight_bytes -= b->bytes;
    }
    s->cv_done.notify_all();
    s->cv_sched.notify_all();
    delete b;
}

// Enqueues one batch on a stream; on failure marks its requests failed.
void launch_batch(fk_server *s, Batch *b) {
    const fk_table *t = s->tables[b->reqs[0]->table];
    const int prec = b->reqs[0]->prec;
    const size_t esz = FK_IO64(prec) ? 8 : 4;
    int R = 0;
    for (Request *r : b->reqs) R += r->R;
    cudaStream_t st = s->streams[b->stream];
    char *dF = nullptr, *dO = nullptr;
    int rc = FK_OK;
    const size_t fb = esz * (size_t)R * NFL * t->nxg, ob = esz * (size_t)R * t->ndata;
    cudaError_t e = take_fault(s, FK_FAULT_DEVICE) ? cudaErrorMemoryAllocation : cudaMallocAsync((void **)&dF, fb, st);
    if (!e) e = cudaMallocAsync((void **)&dO, ob, st);
    if (e) rc = cuda_fail(e, "serve: device buffers");
    size_t off = 0;
    for (Request *r : b->reqs) {
        if (rc) break;
        e = cudaMemcpyAsync(dF + off, r->F, r->f_bytes, cudaMemcpyHostToDevice, st);
        if (e) rc = cuda_fail(e, "serve: H2D");
        off += r->f_bytes;
    }
    if (!rc && take_fault(s, FK_FAULT_LAUNCH)) rc = fail(FK_ECUDA, "serve: convolution launch failed (injected)");
    if (!rc) {
        rc = t->kind == FK_KIND_HAD ? fk_had_conv(t, dF, R, dO, 0, prec, st)
                                    : fk_dis_conv(t, dF, R, dO, 0, prec, st);
    }
    off = 0;
    for (Request *r : b->reqs) {
        if (rc) break;
        e = cudaMemcpyAsync(r->O, dO + off, r->o_bytes, cudaMemcpyDeviceToHost, st);
        if (e) rc = cuda_fail(e, "serve: D2H");
        off += r->o_bytes;
    }
    if (dF) cudaFreeAsync(dF, st);
    if (dO) cudaFreeAsync(dO, st);
    b->t0 = std::chrono::steady_clock::now();
    if (!rc && take_fault(s, FK_FAULT_DROP)) {
        // the completion message is lost: only the watchdog can finish this batch
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (!e) e = cudaEventRecord(ev, st);
        if (e) {
            rc = cuda_fail(e, "serve: completion event");
        } else {
            std::lock_guard<std::mutex> l(s->mu);
            s->unconfirmed.push_back({b, ev});
            s->cv_sched.notify_all();  // the scheduler starts polling for it
            return;
        }
    }
    if (!rc) {
        e = cudaLaunchHostFunc(st, batch_done, b);
        if (e) rc = cuda_fail(e, "serve: completion callback");
    }
    if (rc) {
        // nothing will call back: fail the requests here (the stream is
        // synchronised first so no copy into their buffers is still pending)
        cudaStreamSynchronize(st);
        std::lock_guard<std::mutex> l(s->mu);
        for (Request *r : b->reqs) {
            r->status = rc;
            r->done = true;
        }
        s->inflight--;
        s->inflight_bytes -= b->bytes;
        delete b;
        s->cv_done.notify_all();
    } else {
        std::lock_guard<std::mutex> l(s->mu);
        s->launches++;
    }
}

// Requests are merged only within one kernel class, so that a replica's
// result is the same alone and in any batch: the FP64/FP32 hadronic path
// streams R = 1 and uses the factorised kernel for R >= 2 (DIS: R <= 4 and
// R > 4); each tensor-core precision is a single class.
int kernel_class(const fk_table *t, int prec, int R) {
    if (prec == FK_FP64_TC) return 3;
    if (prec != FK_FP64 && prec != FK_FP32) return 2;
    if (t->kind == FK_KIND_HAD) return R == 1 ? 0 : 1;
    return R <= 4 ? 0 : 1;
}

void scheduler(fk_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> l(s->mu);
    auto ready = [&] { return s->stop || (!s->queue.empty() && s->inflight < s->max_inflight); };
    while (true) {
        while (!ready()) {
            if (has_unconfirmed(s)) {  // poll the lost completions every 10 ms
                s->cv_sched.wait_for(l, std::chrono::milliseconds(10));
                if (reap_unconfirmed(s)) s->cv_done.notify_all();
            } else {
                s->cv_sched.wait(l);
            }
        }
        if (s->stop && s->queue.empty()) break;
        if (s->stop) {
            // what never started is cancelled
            for (Request *r : s->queue) {
                r->status = FK_ECANCELED;
                r->done = true;
            }
            s->queue.clear();
            s->cv_done.notify_all();
            break;
        }
        // head of the queue decides the batch; join later requests on the
        // same table, precision and kernel class while memory allows
        Request *head = s->queue.front();
        const fk_table *t = s->tables[head->table];
        if (s->resident + s->inflight_bytes + head->dev_bytes > s->budget) {
            if (s->inflight == 0) {  // cannot fit even alone (checked at submit)
                head->status = FK_EBUDGET;
                head->done = true;
                s->queue.pop_front();
                s->cv_done.notify_all();
            } else {
                s->cv_sched.wait_for(l, std::chrono::milliseconds(10));
                if (reap_unconfirmed(s)) s->cv_done.notify_all();
            }
            continue;
        }
        Batch *b = new Batch();
        b->srv = s;
        const int cls = kernel_class(t, head->prec, head->R);
        int R = 0;
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            Request *r = *it;
            const int Rn = R + r->R;
            const bool same = r->table == head->table && r->prec == head->prec &&
                              kernel_class(t, r->prec, r->R) == cls && kernel_class(t, r->prec, Rn) == cls;
            const size_t add = request_device_bytes(t, Rn, r->prec) - (R ? request_device_bytes(t, R, r->prec) : 0);
            if (same && (b->reqs.empty() || s->resident + s->inflight_bytes + b->bytes + add <= s->budget)) {
                b->reqs.push_back(r);
                b->bytes += add;
                R = Rn;
                it = s->queue.erase(it);
                if (Rn >= 4096) break;
            } else {
                ++it;
            }
        }
        s->inflight++;
        s->inflight_bytes += b->bytes;
        s->peak_bytes = std::max(s->peak_bytes, s->resident + s->inflight_bytes);
        b->stream = s->next_stream;
        s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
        l.unlock();
        launch_batch(s, b);
        l.lock();
    }
    // wait for the batches in flight (and give up the lost ones)
    while (s->inflight > 0) {
        s->cv_done.wait_for(l, std::chrono::milliseconds(10));
        if (reap_unconfirmed(s)) s->cv_done.notify_all();
    }
}

}  // namespace
}  // namespace fk

extern "C" {

int fk_serve_create(size_t hbm_budget_bytes, int max_inflight, fk_server **out) {
    if (!out || hbm_budget_bytes == 0 || max_inflight < 1)
        return fail(FK_EINVAL, "fk_serve_create: bad budget, max_inflight or out");
    *out = nullptr;
    fk_server *s = new fk_server();
    s->budget = hbm_budget_bytes;
    s->max_inflight = max_inflight;
    cudaGetDevice(&s->device);
    const int ns = std::min(max_inflight, 8);
    for (int i = 0; i < ns; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return fail(FK_ECUDA, "fk_serve_create: stream");
        }
        s->streams.push_back(st);
    }
    // FK_FAULT="kind:count,...": host-side faults armed at creation (kinds
    // pinned, device, launch, drop), as fk_serve_inject
    if (const char *env = std::getenv("FK_FAULT")) {
        std::string spec(env);
        size_t pos = 0;
        while (pos < spec.size()) {
            size_t end = spec.find(',', pos);
            if (end == std::string::npos) end = spec.size();
            const std::string item = spec.substr(pos, end - pos);
            const size_t colon = item.find(':');
            const std::string kind = item.substr(0, colon);
            const int count = colon == std::string::npos ? 1 : std::atoi(item.c_str() + colon + 1);
            const int k = kind == "pinned" ? FK_FAULT_PINNED : kind == "device" ? FK_FAULT_DEVICE
                          : kind == "launch" ? FK_FAULT_LAUNCH : kind == "drop" ? FK_FAULT_DROP : 0;
            if (k && count > 0) s->faults[k] += count;
            pos = end + 1;
        }
    }
    s->worker = std::thread(scheduler, s);
    *out = s;
    return FK_OK;
}

int fk_serve_add_table(fk_server *s, fk_table *t, int *table_id) {
    if (!s || !t || !table_id) return fail(FK_EINVAL, "fk_serve_add_table: null argument");
    if (t->kind == FK_KIND_DENSE) return fail(FK_EUNSUPPORTED, "fk_serve_add_table: the server takes DIS and hadronic tables");
    std::lock_guard<std::mutex> l(s->mu);
    if (s->resident + t->bytes > s->budget) return fail(FK_EBUDGET, "table does not fit the server budget");
    s->tables.push_back(t);
    s->resident += t->bytes;
    s->peak_bytes = std::max(s->peak_bytes, s->resident);
    *table_id = (int)s->tables.size() - 1;
    return FK_OK;
}

int fk_serve_submit(fk_server *s, int table_id, const void *F_host, int R, int prec, uint64_t *ticket) {
    if (!s || !F_host || !ticket || R < 1) return fail(FK_EINVAL, "fk_serve_submit: bad argument");
    if (prec < FK_FP64 || prec > FK_FP64_TC) return fail(FK_EINVAL, "fk_serve_submit: unknown precision");
    fk_table *t;
    {
        std::lock_guard<std::mutex> l(s->mu);
        if (table_id < 0 || table_id >= (int)s->tables.size()) return fail(FK_ENOTFOUND, "unknown table id");
        t = s->tables[table_id];
    }
    if (!(t->mask & FK_PREC_BIT(prec))) return fail(FK_EUNSUPPORTED, "precision not stored in this table");
    auto r = std::make_unique<Request>();
    r->table = table_id;
    r->R = R;
    r->prec = prec;
    const size_t esz = FK_IO64(prec) ? 8 : 4;
    r->f_bytes = esz * (size_t)R * NFL * t->nxg;
    r->o_bytes = esz * (size_t)R * t->ndata;
    r->dev_bytes = request_device_bytes(t, R, prec);
    {
        std::lock_guard<std::mutex> l(s->mu);
        if (s->resident + r->dev_bytes > s->budget)
            return fail(FK_EBUDGET, "request can never fit the server budget");
    }
    size_t c1 = 0, c2 = 0;
    const bool injected = take_fault(s, FK_FAULT_PINNED);
    r->F = injected ? nullptr : s->pinned.get(r->f_bytes, &c1);
    r->O = injected ? nullptr : s->pinned.get(r->o_bytes, &c2);
    if (!r->F || !r->O) {
        s->pinned.put(r->F, c1);
        s->pinned.put(r->O, c2);
        return fail(FK_ENOMEM, "pinned staging");
    }
    std::memcpy(r->F, F_host, r->f_bytes);
    {
        std::lock_guard<std::mutex> l(s->mu);
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        s->queue.push_back(r.get());
        s->reqs.emplace(r->ticket, std::move(r));
    }
    s->cv_sched.notify_one();
    return FK_OK;
}

static int finish(fk_server *s, std::unique_lock<std::mutex> &l, uint64_t ticket, void *O_host) {
    auto it = s->reqs.find(ticket);
    Request *r = it->second.get();
    const int st = r->cancelled && r->status == FK_OK ? FK_ECANCELED : r->status;
    if (st == FK_OK && O_host) std::memcpy(O_host, r->O, r->o_bytes);
    s->pinned.put(r->F, pow2_class(r->f_bytes));
    s->pinned.put(r->O, pow2_class(r->o_bytes));
    s->reqs.erase(it);
    return st;
}

int fk_serve_poll(fk_server *s, uint64_t ticket, void *O_host, int *done) {
    if (!s || !done) return fail(FK_EINVAL, "fk_serve_poll: null argument");
    std::unique_lock<std::mutex> l(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(FK_ENOTFOUND, "unknown ticket");
    if (!it->second->done) {
        *done = 0;
        return FK_EPENDING;
    }
    *done = 1;
    return finish(s, l, ticket, O_host);
}

int fk_serve_wait(fk_server *s, uint64_t ticket, void *O_host, int timeout_ms) {
    if (!s) return fail(FK_EINVAL, "fk_serve_wait: null server");
    std::unique_lock<std::mutex> l(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(FK_ENOTFOUND, "unknown ticket");
    Request *r = it->second.get();
    const bool ok = s->cv_done.wait_for(l, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                        [&] { return r->done; });
    if (!ok) return fail(FK_EPENDING, "request still running after the wait");
    return finish(s, l, ticket, O_host);
}

int fk_serve_cancel(fk_server *s, uint64_t ticket) {
    if (!s) return fail(FK_EINVAL, "fk_serve_cancel: null server");
    std::lock_guard<std::mutex> l(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(FK_ENOTFOUND, "unknown ticket");
    Request *r = it->second.get();
    if (r->done) return FK_OK;  // finished already: its result stands
    auto q = std::find(s->queue.begin(), s->queue.end(), r);
    if (q != s->queue.end()) {  // not started: it never will
        s->queue.erase(q);
        r->status = FK_ECANCELED;
        r->done = true;
        s->cv_done.notify_all();
    } else {
        r->cancelled = true;  // running: its result will be discarded
    }
    return FK_OK;
}

int fk_serve_inject(fk_server *s, int fault, int count) {
    if (!s || fault < FK_FAULT_PINNED || fault > FK_FAULT_DROP || count < 0)
        return fail(FK_EINVAL, "fk_serve_inject: bad server, fault kind or count");
    std::lock_guard<std::mutex> l(s->mu);
    s->faults[fault] = count;
    return FK_OK;
}

int fk_serve_stats(const fk_server *cs, uint64_t *completed, uint64_t *dp_rep, uint64_t *launches,
                   size_t *peak_bytes, int *queued) {
    if (!cs) return fail(FK_EINVAL, "fk_serve_stats: null server");
    fk_server *s = const_cast<fk_server *>(cs);
    std::lock_guard<std::mutex> l(s->mu);
    if (completed) *completed = s->completed;
    if (dp_rep) *dp_rep = s->dp_rep;
    if (launches) *launches = s->launches;
    if (peak_bytes) *peak_bytes = s->peak_bytes;
    if (queued) *queued = (int)s->queue.size();
    return FK_OK;
}

int fk_serve_destroy(fk_server *s) {
    if (!s) return FK_OK;
    {
        std::lock_guard<std::mutex> l(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto &kv : s->reqs) {
        s->pinned.put(kv.second->F, pow2_class(kv.second->f_bytes));
        s->pinned.put(kv.second->O, pow2_class(kv.second->o_bytes));
    }
    s->reqs.clear();
    delete s;
    return FK_OK;
}

}  // extern "C"
