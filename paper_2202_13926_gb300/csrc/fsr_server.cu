// Serving form: a worker thread that admits queued requests into a device
// memory pool, batches every admitted request into the next launch of the
// batch kernel, and overlaps copies in, launches and copies out of different
// requests on separate streams.  Contract: include/fsr.h (fsr_server_*).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "fsr.h"
#include "fsr_internal.h"
#include "fsr_launch.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kAlign = 256;
constexpr int kMaxBatch = 256;   // requests per launch at most
// Requests of at most this many pixels (1080p and smaller) are the short
// class: launched on the high-priority stream of slot 0.
constexpr long long kShortPixels = 1920ll * 1088ll;
// S = 32 launches of the long class run short-lived CTAs (a warp takes one
// chunk of kShortChunk blocks), so that the CTAs of a short-class launch
// (persistent, high priority) are scheduled as soon as CTAs of a running
// long launch finish.
constexpr int kShortChunk = 4;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Pool range of one request: image (4 B/px), mask (1 B/px), output (4 B/px).
size_t mask_offset(size_t npix) { return align_up(npix * 4); }
size_t out_offset(size_t npix) { return align_up(npix * 4) + align_up(npix); }
size_t request_bytes(size_t npix) { return out_offset(npix) + align_up(npix * 4); }

// First-fit allocator over [0, size) of the device pool, free ranges coalesced.
class PoolAllocator {
public:
    explicit PoolAllocator(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off) {
        bytes = align_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                if (used_ > peak_) peak_ = used_;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t peak() const { return peak_; }
    size_t size() const { return size_; }

private:
    size_t size_, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

enum class St { Queued, Admitted, Launched, CopyingOut };

struct Request {
    long long ticket = 0;
    const float* h_img = nullptr;
    const uint8_t* h_mask = nullptr;
    float* h_out = nullptr;
    int H = 0, W = 0, K = 0;
    size_t off = 0, bytes = 0;        // pool range: image, mask, output
    Clock::time_point t_submit;
    cudaEvent_t ev = nullptr;         // copy-in done, later copy-out done
    St st = St::Queued;
    bool failed = false;
};

struct Launch {
    cudaEvent_t done = nullptr;
    std::vector<Request*> reqs;
    size_t table_off = 0, table_bytes = 0;
    int slot = 0;
    bool active = false;
};

}  // namespace

struct fsr_server {
    fsr_handle* h = nullptr;
    fsr_params p{};
    int max_inflight = 1;
    int nstreams = 1;
    unsigned char* pool = nullptr;
    PoolAllocator* alloc = nullptr;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    std::vector<cudaStream_t> s_comp;
    std::vector<void*> h_tables;      // pinned table staging, one per compute slot
    std::vector<Launch> launches;     // one per compute slot
    std::vector<cudaEvent_t> free_events;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;                    // submitted, not admitted
    std::vector<Request*> admitted;                // copy in issued, not launched
    std::vector<Request*> out_pending;             // copy out issued
    std::deque<std::pair<long long, double>> done; // completions not yet polled
    std::thread worker;
    bool stopping = false;
    long long next_ticket = 0, submitted = 0, completed = 0, n_launches = 0;
    int inflight = 0;
};

namespace {

cudaEvent_t take_event(fsr_server* s) {
    if (!s->free_events.empty()) {
        cudaEvent_t e = s->free_events.back();
        s->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

void finish(fsr_server* s, Request* r, Clock::time_point now) {
    const double ms = r->failed ? -1.0 : std::chrono::duration<double, std::milli>(now - r->t_submit).count();
    s->alloc->release(r->off, r->bytes);
    if (r->ev) s->free_events.push_back(r->ev);
    s->done.emplace_back(r->ticket, ms);
    s->completed += 1;
    s->inflight -= 1;
    delete r;
}

// Launches up to kMaxBatch of the requests in q (taken from its front) as
// one batch on the given free slot; the rest stay in q.  A long-class
// request fills the GPU on its own, so the long class launches one request
// at a time in arrival order: the earliest finishes first instead of every
// request of a batch finishing with the batch's last block.  Returns false
// when the launch table does not fit in the pool now (nothing launched).
bool launch_on(fsr_server* s, int slot, std::vector<Request*>& q, bool long_class) {
    const int n = (int)std::min<size_t>(q.size(), long_class ? 1 : kMaxBatch);
    Launch& L = s->launches[slot];
    size_t toff = 0;
    const size_t tbytes = fsri::table_bytes(n);
    if (!s->alloc->alloc(tbytes, &toff)) return false;
    std::vector<Request*> batch(q.begin(), q.begin() + n);
    q.erase(q.begin(), q.begin() + n);
    std::vector<fsr_image_desc> d(n);
    for (int j = 0; j < n; ++j) {
        Request* r = batch[j];
        const size_t npix = (size_t)r->H * r->W;
        d[j].img = reinterpret_cast<const float*>(s->pool + r->off);
        d[j].mask = s->pool + r->off + mask_offset(npix);
        d[j].out = reinterpret_cast<float*>(s->pool + r->off + out_offset(npix));
        d[j].height = r->H;
        d[j].width = r->W;
        d[j].pitch = r->W;
        d[j].iters = r->K;
        d[j].seq_out = nullptr;
    }
    // (errors go to this thread's own record, not to the handle the caller uses)
    const long long total = fsri::build_table(nullptr, n, d.data(), &s->p, s->h_tables[slot]);
    cudaStream_t cs = s->s_comp[slot];
    cudaError_t e = total < 0 ? cudaErrorInvalidValue : cudaSuccess;
    for (Request* r : batch)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, r->ev, 0);
    void* dt = s->pool + toff;
    if (e == cudaSuccess) e = cudaMemcpyAsync(dt, s->h_tables[slot], tbytes, cudaMemcpyHostToDevice, cs);
    const fsrk::Schedule sc = s->h->sched[s->p.precision][fsri::b_index(s->p.block)];
    if (e == cudaSuccess) {
        const bool short_ctas = long_class && s->p.block + 2 * s->p.border == fsrk::S;
        fsrk::BatchArgs a = fsri::batch_args(s->h, dt, n, total, &s->p, short_ctas ? kShortChunk : sc.chunk);
        a.one_round = short_ctas ? 1 : 0;
        e = fsri::launch_batch(a, &s->p, sc, s->h->sm_count, cs);
    }
    if (e == cudaSuccess) e = cudaEventRecord(L.done, cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (Request* r : batch) r->failed = true;
        cudaEventRecord(L.done, cs);
    }
    for (Request* r : batch) r->st = St::Launched;
    L.reqs = batch;
    L.table_off = toff;
    L.table_bytes = tbytes;
    L.active = true;
    s->n_launches += 1;
    return true;
}

// One pass of the worker over completions, admissions and launches (lock held).
bool step(fsr_server* s) {
    bool progressed = false;
    const auto now = Clock::now();
    // 1. copies out that finished: the request is complete
    for (size_t i = 0; i < s->out_pending.size();) {
        Request* r = s->out_pending[i];
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        if (q != cudaSuccess) r->failed = true;
        s->out_pending[i] = s->out_pending.back();
        s->out_pending.pop_back();
        finish(s, r, now);
        progressed = true;
    }
    // 2. launches that finished: copy their outputs back
    for (Launch& L : s->launches) {
        if (!L.active) continue;
        const cudaError_t q = cudaEventQuery(L.done);
        if (q == cudaErrorNotReady) continue;
        if (cudaStreamWaitEvent(s->s_out, L.done, 0) != cudaSuccess) cudaGetLastError();
        for (Request* r : L.reqs) {
            if (q != cudaSuccess) r->failed = true;
            cudaError_t e = cudaMemcpyAsync(r->h_out, s->pool + r->off + out_offset((size_t)r->H * r->W),
                                            (size_t)r->H * r->W * sizeof(float), cudaMemcpyDeviceToHost, s->s_out);
            if (e == cudaSuccess) e = cudaEventRecord(r->ev, s->s_out);
            if (e != cudaSuccess) {
                cudaGetLastError();
                r->failed = true;
            }
            r->st = St::CopyingOut;
            s->out_pending.push_back(r);
        }
        s->alloc->release(L.table_off, L.table_bytes);
        L.reqs.clear();
        L.active = false;
        progressed = true;
    }
    // 3. admission in arrival order while the pool and the slots allow
    while (!s->queue.empty() && s->inflight < s->max_inflight) {
        Request* r = s->queue.front();
        size_t off = 0;
        if (!s->alloc->alloc(r->bytes, &off)) break;
        r->off = off;
        r->ev = take_event(s);
        const size_t npix = (size_t)r->H * r->W;
        cudaError_t e = r->ev ? cudaSuccess : cudaErrorMemoryAllocation;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->pool + off, r->h_img, npix * sizeof(float), cudaMemcpyHostToDevice, s->s_in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->pool + off + mask_offset(npix), r->h_mask, npix, cudaMemcpyHostToDevice, s->s_in);
        if (e == cudaSuccess) e = cudaEventRecord(r->ev, s->s_in);
        if (e != cudaSuccess) {
            cudaGetLastError();
            r->failed = true;
        }
        s->queue.pop_front();
        s->inflight += 1;
        r->st = St::Admitted;
        s->admitted.push_back(r);
        progressed = true;
    }
    // 4. launch the admitted requests (continuous batching): the short class
    //    on slot 0 (high-priority stream), the long class on the other slots
    //    (one slot: everything on slot 0)
    if (!s->admitted.empty()) {
        std::vector<Request*> shortq, longq;
        for (Request* r : s->admitted) {
            if (r->failed) {
                r->st = St::CopyingOut;
                s->out_pending.push_back(r);
            } else if ((long long)r->H * r->W <= kShortPixels) {
                shortq.push_back(r);
            } else {
                longq.push_back(r);
            }
        }
        s->admitted.clear();
        auto free_slot = [&](bool allow0, bool allow_rest) {
            if (allow0 && !s->launches[0].active) return 0;
            if (allow_rest)
                for (int i = 1; i < s->nstreams; ++i)
                    if (!s->launches[i].active) return i;
            return -1;
        };
        const bool many = s->nstreams > 1;
        // what is not launched now (no free slot, no room for the table, or
        // beyond kMaxBatch) waits in the admitted list for the next pass
        if (!shortq.empty()) {
            const int slot = free_slot(true, !many);
            if (slot >= 0 && launch_on(s, slot, shortq, false)) progressed = true;
            s->admitted.insert(s->admitted.end(), shortq.begin(), shortq.end());
        }
        if (!longq.empty()) {
            const int slot = free_slot(!many, many);
            if (slot >= 0 && launch_on(s, slot, longq, true)) progressed = true;
            s->admitted.insert(s->admitted.end(), longq.begin(), longq.end());
        }
    }
    return progressed;
}

void worker_main(fsr_server* s) {
    cudaSetDevice(s->h->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        const bool progressed = step(s);
        if (progressed) s->cv_done.notify_all();
        const bool busy = !s->queue.empty() || !s->admitted.empty() || !s->out_pending.empty() ||
                          std::any_of(s->launches.begin(), s->launches.end(), [](const Launch& L) { return L.active; });
        if (s->stopping && !busy) break;
        if (!progressed) {
            // device work in flight: poll again shortly; idle: sleep until a submission
            if (busy) s->cv_work.wait_for(lk, std::chrono::microseconds(50));
            else s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

}  // namespace

extern "C" {

int fsr_server_create(fsr_handle* h, const fsr_server_config* cfg, const fsr_params* p, fsr_server** out) {
    if (!h) return fsri::fail(nullptr, FSR_ERR_INVALID_ARG, "handle is NULL");
    if (!cfg || !out) return fsri::fail(h, FSR_ERR_INVALID_ARG, "cfg and out must be non-NULL");
    *out = nullptr;
    int r = fsri::check_method(h, p);
    if (r != FSR_OK) return r;
    if (p->precision != FSR_FP32 && p->precision != FSR_FP64_DEBUG)
        return fsri::fail(h, FSR_ERR_UNSUPPORTED, "the server runs FSR_FP32 or FSR_FP64_DEBUG");
    if (p->reuse > 0.f)
        return fsri::fail(h, FSR_ERR_UNSUPPORTED, "re-use of reconstructed pixels runs in the single-image entry points");
    if (cfg->pool_bytes < (1u << 20) || cfg->max_inflight < 1 || cfg->streams < 1 || cfg->streams > 8)
        return fsri::fail(h, FSR_ERR_INVALID_ARG, "pool_bytes >= 1 MiB, max_inflight >= 1 and 1 <= streams <= 8");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    fsr_server* s = new (std::nothrow) fsr_server();
    if (!s) return fsri::fail(h, FSR_ERR_OOM, "host allocation of the server failed");
    s->h = h;
    s->p = *p;
    s->p.seq_out = nullptr;
    s->max_inflight = cfg->max_inflight;
    s->nstreams = cfg->streams;
    cudaError_t e = cudaMalloc(&s->pool, cfg->pool_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        cudaSetDevice(prev);
        return fsri::fail(h, FSR_ERR_OOM, "cudaMalloc of the %zu-byte pool: %s", cfg->pool_bytes, cudaGetErrorString(e));
    }
    s->alloc = new PoolAllocator(cfg->pool_bytes);
    bool okk = cudaStreamCreateWithFlags(&s->s_in, cudaStreamNonBlocking) == cudaSuccess &&
               cudaStreamCreateWithFlags(&s->s_out, cudaStreamNonBlocking) == cudaSuccess;
    s->s_comp.resize(s->nstreams, nullptr);
    s->h_tables.resize(s->nstreams, nullptr);
    s->launches.resize(s->nstreams);
    int prio_low = 0, prio_high = 0;   // numerically lower = higher priority
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        cudaGetLastError();
        prio_low = prio_high = 0;
    }
    for (int i = 0; i < s->nstreams && okk; ++i) {
        okk = cudaStreamCreateWithPriority(&s->s_comp[i], cudaStreamNonBlocking, i == 0 ? prio_high : prio_low) ==
                  cudaSuccess &&
              cudaMallocHost(&s->h_tables[i], fsri::table_bytes(kMaxBatch)) == cudaSuccess &&
              cudaEventCreateWithFlags(&s->launches[i].done, cudaEventDisableTiming) == cudaSuccess;
        s->launches[i].slot = i;
    }
    cudaSetDevice(prev);
    if (!okk) {
        cudaGetLastError();
        fsr_server_destroy(s);
        return fsri::fail(h, FSR_ERR_CUDA, "creating the server's streams and buffers failed");
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    h->err[0] = 0;
    return FSR_OK;
}

int fsr_server_submit(fsr_server* s, const float* img, const uint8_t* mask, int height, int width, int iters,
                      float* out, long long* ticket) {
    if (!s) return fsri::fail(nullptr, FSR_ERR_INVALID_ARG, "server is NULL");
    if (!img || !mask || !out || height <= 0 || width <= 0 || iters < 0 || iters > 65535)
        return fsri::fail(s->h, FSR_ERR_INVALID_ARG, "bad request: pointers, size %d x %d or iters %d", height, width,
                          iters);
    const size_t npix = (size_t)height * width;
    const size_t bytes = request_bytes(npix);
    if (bytes + align_up(fsri::table_bytes(1)) > s->alloc->size())
        return fsri::fail(s->h, FSR_ERR_INVALID_ARG, "a %d x %d request needs %zu bytes, more than the pool (%zu)",
                          height, width, bytes, s->alloc->size());
    Request* r = new (std::nothrow) Request();
    if (!r) return fsri::fail(s->h, FSR_ERR_OOM, "host allocation of a request failed");
    r->h_img = img;
    r->h_mask = mask;
    r->h_out = out;
    r->H = height;
    r->W = width;
    r->K = iters;
    r->bytes = bytes;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) {
            delete r;
            return fsri::fail(s->h, FSR_ERR_INVALID_ARG, "server is stopping");
        }
        r->ticket = s->next_ticket++;
        s->submitted += 1;
        s->queue.push_back(r);
        if (ticket) *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return FSR_OK;
}

int fsr_server_poll(fsr_server* s, long long* tickets, double* latency_ms, int max, int* n, int wait_ms) {
    if (!s || !n || max < 0) return fsri::fail(nullptr, FSR_ERR_INVALID_ARG, "bad poll arguments");
    std::unique_lock<std::mutex> lk(s->mu);
    if (wait_ms > 0 && s->done.empty())
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
    int k = 0;
    while (k < max && !s->done.empty()) {
        if (tickets) tickets[k] = s->done.front().first;
        if (latency_ms) latency_ms[k] = s->done.front().second;
        s->done.pop_front();
        ++k;
    }
    *n = k;
    return FSR_OK;
}

int fsr_server_stats(const fsr_server* s, long long* submitted, long long* completed, int* queued, int* inflight,
                     long long* launches, size_t* peak_pool_bytes) {
    if (!s) return FSR_ERR_INVALID_ARG;
    fsr_server* m = const_cast<fsr_server*>(s);
    std::lock_guard<std::mutex> lk(m->mu);
    if (submitted) *submitted = s->submitted;
    if (completed) *completed = s->completed;
    if (queued) *queued = (int)s->queue.size();
    if (inflight) *inflight = s->inflight;
    if (launches) *launches = s->n_launches;
    if (peak_pool_bytes) *peak_pool_bytes = s->alloc ? s->alloc->peak() : 0;
    return FSR_OK;
}

int fsr_server_destroy(fsr_server* s) {
    if (!s) return FSR_OK;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stopping = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->h->device);
    for (cudaStream_t c : s->s_comp)
        if (c) cudaStreamSynchronize(c);
    if (s->s_in) cudaStreamSynchronize(s->s_in);
    if (s->s_out) cudaStreamSynchronize(s->s_out);
    for (cudaStream_t c : s->s_comp)
        if (c) cudaStreamDestroy(c);
    if (s->s_in) cudaStreamDestroy(s->s_in);
    if (s->s_out) cudaStreamDestroy(s->s_out);
    for (void* t : s->h_tables)
        if (t) cudaFreeHost(t);
    for (Launch& L : s->launches)
        if (L.done) cudaEventDestroy(L.done);
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    cudaFree(s->pool);
    delete s->alloc;
    cudaSetDevice(prev);
    delete s;
    return FSR_OK;
}

}  // extern "C"
