// Serving: continuous batching of channelisation requests.
//
// A request is one chunk of one stream.  Each stream keeps its filter state on
// the device -- the last T-1 frames of raw input -- so that a chunk sees
// state ++ chunk as its frame sequence and the concatenated outputs equal the
// single-pass channeliser on the concatenated input (spectra are the "valid"
// outputs of Sec. 5.2's per-branch FIR).  State lives in two device buffers
// per stream (read one, write the other).
//
// Scheduling (host worker thread): at every step it polls the batches on the
// device and forms the next batch from the queue, in submission order, while
// fewer than max_slots requests are on the device and the bytes they pin
// (input and output buffers) fit the HBM budget next to the resident state of
// the open streams.  A batch is one kernel launch per kernel variant over all
// its streams (the persistent launch of pfb_execute_batch), one batched state
// update and one event.  Consecutive chunks of a stream whose input and output
// buffers continue each other merge into one descriptor; any other chunk of a
// stream already in the batch waits for a later batch.  Batches rotate over a
// small pool of CUDA streams and wait (cudaStreamWaitEvent) on the previous
// batch of each of their streams, so independent work overlaps on the device
// while each stream's chunks run in order.  Requests that arrive while others
// run join the next batch.  Latency is submit -> observed completion (the
// batch event, polled every few microseconds).  A request not seen complete
// within timeout_ms reports PFB_ERR_TIMEOUT; its slot stays held until the
// device finishes it.
//
// Host-side fault injection for tests (no GPU fault is ever provoked):
//   PFB_FAULT=launch_fail:<k>      the k-th request taken into a batch is not
//                                  launched and fails with PFB_ERR_CUDA (later
//                                  chunks of its stream fail too);
//   PFB_FAULT=lose_completion:<k>  the k-th launched request's completion is
//                                  never observed, so it times out.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <thread>

#include "internal.h"

namespace pfb {

using Clock = std::chrono::steady_clock;

// new_state[i] = frame (old_frames + chunk_frames - n_keep + i) of (state ++ chunk),
// for up to kMaxStateUpdates streams per launch (one block row per stream)
struct StateUpdate {
    const uint2 *old_state;
    const uint2 *chunk;
    uint2 *new_state;
    int64_t old_frames, chunk_frames, n_keep, words_per_frame;
};
constexpr int kMaxStateUpdates = 64;
struct StateUpdateArgs {
    StateUpdate u[kMaxStateUpdates];
    int n;
};

__global__ void k_state_update(const __grid_constant__ StateUpdateArgs a) {
    const StateUpdate &u = a.u[blockIdx.y];
    const int64_t total = u.n_keep * u.words_per_frame;
    const int64_t first = u.old_frames + u.chunk_frames - u.n_keep;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = w / u.words_per_frame, off = w - i * u.words_per_frame;
        const int64_t g = first + i;
        u.new_state[w] = (g < u.old_frames) ? u.old_state[g * u.words_per_frame + off]
                                            : u.chunk[(g - u.old_frames) * u.words_per_frame + off];
    }
}

static pfb_status launch_state_updates(const std::vector<StateUpdate> &ups, cudaStream_t stream) {
    for (size_t g0 = 0; g0 < ups.size(); g0 += kMaxStateUpdates) {
        StateUpdateArgs a;
        std::memset(&a, 0, sizeof(a));
        int64_t maxw = 0;
        for (size_t i = g0; i < ups.size() && a.n < kMaxStateUpdates; ++i) {
            if (ups[i].n_keep <= 0) continue;
            a.u[a.n++] = ups[i];
            maxw = std::max(maxw, ups[i].n_keep * ups[i].words_per_frame);
        }
        if (a.n == 0) continue;
        const int threads = 256;
        const unsigned bx = (unsigned)std::min<int64_t>((maxw + threads - 1) / threads, 64);
        k_state_update<<<dim3(bx, a.n), threads, 0, stream>>>(a);
        g_launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "launch k_state_update");
    }
    return PFB_OK;
}

pfb_status launch_state_update(const void *old_state, int64_t old_frames, const void *chunk, int64_t chunk_frames,
                               void *new_state, int64_t n_keep, int64_t frame_bytes, cudaStream_t stream) {
    StateUpdate u{static_cast<const uint2 *>(old_state), static_cast<const uint2 *>(chunk),
                  static_cast<uint2 *>(new_state), old_frames, chunk_frames, n_keep, frame_bytes / 8};
    return launch_state_updates({u}, stream);
}

struct Batch;

struct Request {
    int64_t ticket = 0, stream_id = 0;
    const void *d_chunk = nullptr;
    void *d_out = nullptr;
    int64_t n_samples = 0, S = 0, bytes = 0;
    pfb_status status = PFB_PENDING;
    bool launched = false, lost = false, released = false;
    Batch *batch = nullptr;
    Clock::time_point t_submit, t_launch, t_done;
};

struct PStream {
    int64_t id = 0;
    Plan *plan = nullptr;
    void *state[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t state_frames = 0;       // valid frames in state[cur] at the next launch
    int64_t frames_submitted = 0;   // frames of all chunks submitted so far
    int64_t state_bytes = 0;
    int64_t outstanding = 0;        // submitted and not finished
    bool failed = false;            // an earlier chunk failed: later chunks fail too
    bool closing = false;
    cudaEvent_t last_event = nullptr;  // event of the last batch that advanced this stream
    int last_cs = -1;                  // CUDA stream that batch ran on
};

// A batch: every request admitted at one scheduling step, run as one launch
// per kernel variant plus one batched state update, completing on one event.
struct Batch {
    std::vector<Request *> reqs;
    cudaEvent_t done = nullptr;
    int err_idx = -1;                // this batch's kernel error word (server pool)
    int cs = 0;
    Clock::time_point t_launch;
    bool device_done = false;
};

struct Server {
    pfb_server_desc desc;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> free_events;
    // kernel error words, one per batch in flight (mapped, pinned host memory)
    static constexpr int kErrWords = 256;
    int *h_err = nullptr, *d_err = nullptr;
    std::vector<int> free_err;
    std::map<int64_t, std::unique_ptr<PStream>> streams;
    std::map<int64_t, std::unique_ptr<Request>> tickets;
    std::deque<Request *> queue;             // submitted, not launched (submission order)
    std::vector<std::unique_ptr<Batch>> batches;  // launched, device completion not seen
    int64_t inflight = 0;                    // requests launched and still holding a slot
    int next_cs = 0;
    int64_t next_stream = 1, next_ticket = 1;
    int64_t reserved = 0, peak_reserved = 0;
    int64_t n_submitted = 0, n_completed = 0, n_failed = 0, n_rejected = 0, samples_completed = 0;
    int64_t n_batches = 0, n_batched_requests = 0;
    std::vector<double> latencies_us;
    int64_t launch_attempts = 0, launches_done = 0;
    int64_t fault_launch_fail = -1, fault_lose = -1;
};

static void parse_faults(Server &s) {
    const char *f = std::getenv("PFB_FAULT");
    if (!f) return;
    std::string v(f);
    auto num = [&](const std::string &key) -> int64_t {
        size_t p = v.find(key + ":");
        if (p == std::string::npos) return -1;
        return std::atoll(v.c_str() + p + key.size() + 1);
    };
    s.fault_launch_fail = num("launch_fail");
    s.fault_lose = num("lose_completion");
}

static void finish(Server &s, Request &r, pfb_status st) {
    r.status = st;
    r.t_done = Clock::now();
    PStream &ps = *s.streams.at(r.stream_id);
    ps.outstanding--;
    if (st == PFB_OK) {
        s.n_completed++;
        s.samples_completed += r.n_samples;
        s.latencies_us.push_back(std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count());
    } else {
        s.n_failed++;
        if (st != PFB_ERR_TIMEOUT) ps.failed = true;
    }
}

static cudaEvent_t get_event(Server &s) {
    if (!s.free_events.empty()) {
        cudaEvent_t e = s.free_events.back();
        s.free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

// Form and launch one batch from the queue (mutex held).  Requests are taken
// in submission order while slots and budget allow; a stream contributes one
// run of chunks whose input and output buffers continue each other (merged
// into one descriptor); a chunk that does not continue the run waits for a
// later batch, so each stream's chunks run in submission order.
static void launch_batch(Server &s) {
    if (s.queue.empty()) return;
    std::vector<Request *> picked;
    std::map<int64_t, Request *> tail;   // last picked request of each stream
    std::map<int64_t, bool> blocked;
    int64_t bytes = 0;
    for (size_t i = 0; i < s.queue.size(); ++i) {
        Request *r = s.queue[i];
        if (blocked[r->stream_id]) continue;
        if (s.inflight + (int64_t)picked.size() >= s.desc.max_slots) break;
        if (s.reserved + bytes + r->bytes > s.desc.hbm_budget_bytes) break;
        auto t = tail.find(r->stream_id);
        if (t != tail.end()) {
            const Request *p = t->second;
            const PStream &ps = *s.streams.at(r->stream_id);
            const char *in_end = static_cast<const char *>(p->d_chunk) + p->n_samples * ps.plan->esize;
            const float2 *out_end = static_cast<const float2 *>(p->d_out) + p->S * ps.plan->P;
            const bool cont = in_end == static_cast<const char *>(r->d_chunk) &&
                              (r->S == 0 || p->S == 0 || out_end == static_cast<const float2 *>(r->d_out));
            if (!cont) {
                blocked[r->stream_id] = true;
                continue;
            }
        }
        picked.push_back(r);
        tail[r->stream_id] = r;
        bytes += r->bytes;
    }
    if (picked.empty()) return;
    for (Request *r : picked) {
        auto it = std::find(s.queue.begin(), s.queue.end(), r);
        s.queue.erase(it);
    }
    // injected launch failures, and streams that already failed
    std::vector<Request *> go;
    for (Request *r : picked) {
        s.launch_attempts++;
        PStream &ps = *s.streams.at(r->stream_id);
        if (s.launch_attempts == s.fault_launch_fail) {
            finish(s, *r, fail(PFB_ERR_CUDA, "injected launch failure"));
        } else if (ps.failed) {
            finish(s, *r, fail(PFB_ERR_CUDA, "an earlier chunk of this stream failed"));
        } else {
            go.push_back(r);
        }
    }
    if (go.empty()) return;
    auto b = std::make_unique<Batch>();
    b->cs = s.next_cs++ % (int)s.pool.size();
    cudaStream_t cs = s.pool[b->cs];
    b->t_launch = Clock::now();
    // order after the previous batch of every stream in this one
    std::vector<cudaEvent_t> waited;
    for (Request *r : go) {
        PStream &ps = *s.streams.at(r->stream_id);
        if (ps.last_event && ps.last_cs != b->cs &&
            std::find(waited.begin(), waited.end(), ps.last_event) == waited.end()) {
            cudaStreamWaitEvent(cs, ps.last_event, 0);
            waited.push_back(ps.last_event);
        }
    }
    // one descriptor per stream run, one launch per plan
    std::map<Plan *, std::vector<StreamDesc>> groups;
    std::vector<StateUpdate> ups;
    std::map<int64_t, std::vector<Request *>> runs;
    std::vector<int64_t> order;
    for (Request *r : go) {
        if (runs.find(r->stream_id) == runs.end()) order.push_back(r->stream_id);
        runs[r->stream_id].push_back(r);
    }
    pfb_status st = PFB_OK;
    for (int64_t sid : order) {
        PStream &ps = *s.streams.at(sid);
        Plan &plan = *ps.plan;
        const auto &rr = runs[sid];
        int64_t F = 0, S = 0;
        for (Request *r : rr) {
            F += r->n_samples / plan.P;
            S += r->S;
        }
        const int64_t n_frames = ps.state_frames + F;
        if (S > 0) {
            StreamDesc d;
            std::memset(&d, 0, sizeof(d));
            d.in = rr.front()->d_chunk;
            d.state = ps.state[ps.cur];
            // the run's output starts at its first chunk that emits spectra
            for (Request *r : rr)
                if (r->S > 0) {
                    d.out = static_cast<float2 *>(r->d_out);
                    break;
                }
            d.n_state = ps.state_frames;
            d.n_frames = n_frames;
            d.S = S;
            d.ldo = plan.P;
            d.taps = family_taps(plan);
            d.scale = plan.desc.in_scale;
            d.T = plan.T;
            groups[&plan].push_back(d);
        }
        const int64_t keep = std::min<int64_t>(plan.T - 1, n_frames);
        ups.push_back(StateUpdate{static_cast<const uint2 *>(ps.state[ps.cur]), static_cast<const uint2 *>(rr.front()->d_chunk),
                                  static_cast<uint2 *>(ps.state[ps.cur ^ 1]), ps.state_frames, F, keep,
                                  (int64_t)plan.P * plan.esize / 8});
        ps.cur ^= 1;
        ps.state_frames = keep;
    }
    if (s.free_err.empty()) st = fail(PFB_ERR_INTERNAL, "no free kernel error word");
    else {
        b->err_idx = s.free_err.back();
        s.free_err.pop_back();
        s.h_err[b->err_idx] = KERR_NONE;
    }
    for (auto &g : groups) {
        if (st == PFB_OK)
            st = launch_family(*g.first, g.second.data(), (int)g.second.size(), cs, s.d_err + b->err_idx);
    }
    if (st == PFB_OK) st = launch_state_updates(ups, cs);
    b->done = get_event(s);
    if (st == PFB_OK && (!b->done || cudaEventRecord(b->done, cs) != cudaSuccess)) st = fail(PFB_ERR_CUDA, "event record");
    if (st != PFB_OK) {
        for (Request *r : go) finish(s, *r, st);
        if (b->done) s.free_events.push_back(b->done);
        if (b->err_idx >= 0) {
            // a launch may have gone out before the failure: the word is
            // reused only once the device has finished that launch
            cudaStreamSynchronize(cs);
            s.free_err.push_back(b->err_idx);
        }
        return;
    }
    for (int64_t sid : order) {
        PStream &ps = *s.streams.at(sid);
        ps.last_event = b->done;
        ps.last_cs = b->cs;
    }
    for (Request *r : go) {
        r->launched = true;
        r->batch = b.get();
        r->t_launch = b->t_launch;
        s.launches_done++;
        if (s.launches_done == s.fault_lose) r->lost = true;
        s.reserved += r->bytes;
        s.inflight++;
        b->reqs.push_back(r);
    }
    s.peak_reserved = std::max(s.peak_reserved, s.reserved);
    s.n_batches++;
    s.n_batched_requests += (int64_t)go.size();
    s.batches.push_back(std::move(b));
}

static void poll_inflight(Server &s) {
    const auto now = Clock::now();
    for (size_t i = 0; i < s.batches.size();) {
        Batch &b = *s.batches[i];
        if (!b.device_done) {
            cudaError_t q = cudaEventQuery(b.done);
            if (q == cudaSuccess) {
                b.device_done = true;
                // a kernel of the batch whose bounded wait ran out wrote its
                // error word: the batch's spectra are not valid
                const pfb_status kst = take_kernel_error(s.h_err + b.err_idx, "batch kernel");
                if (kst != PFB_OK)
                    for (Request *r : b.reqs)
                        if (r->status == PFB_PENDING && !r->lost) finish(s, *r, kst);
            } else if (q != cudaErrorNotReady) {
                cudaGetLastError();
                b.device_done = true;
                for (Request *r : b.reqs)
                    if (r->status == PFB_PENDING && !r->lost) finish(s, *r, PFB_ERR_CUDA);
            }
        }
        bool all_released = true;
        for (Request *r : b.reqs) {
            if (r->status == PFB_PENDING) {
                if (b.device_done && !r->lost) {
                    finish(s, *r, PFB_OK);
                } else if (std::chrono::duration<double, std::milli>(now - r->t_launch).count() > s.desc.timeout_ms) {
                    finish(s, *r, PFB_ERR_TIMEOUT);
                }
            }
            // slots and budget are released once the device is done with the
            // request (a request whose completion was lost keeps holding them)
            if (!r->released && b.device_done && !r->lost) {
                r->released = true;
                s.reserved -= r->bytes;
                s.inflight--;
            }
            if (!r->released) all_released = false;
        }
        if (b.device_done && all_released) {
            for (auto &kv : s.streams)
                if (kv.second->last_event == b.done) kv.second->last_event = nullptr;
            s.free_events.push_back(b.done);
            if (b.err_idx >= 0) s.free_err.push_back(b.err_idx);
            s.batches[i] = std::move(s.batches.back());
            s.batches.pop_back();
        } else {
            ++i;
        }
    }
}

static void worker_loop(Server *sp) {
    Server &s = *sp;
    cudaSetDevice(s.device);
    std::unique_lock<std::mutex> lk(s.mu);
    while (!s.stop) {
        if (s.batches.empty() && s.queue.empty()) {
            s.cv_work.wait(lk, [&] { return s.stop || !s.batches.empty() || !s.queue.empty(); });
            continue;
        }
        const int64_t before = s.n_completed + s.n_failed;
        poll_inflight(s);
        launch_batch(s);
        if (s.n_completed + s.n_failed != before) s.cv_done.notify_all();
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(2));
        lk.lock();
    }
}

}  // namespace pfb

using namespace pfb;

extern "C" pfb_status pfb_server_create(const pfb_server_desc *desc, pfb_server_t *out_server) {
    clear_error();
    if (!out_server) return fail(PFB_ERR_INVALID, "out_server is NULL");
    *out_server = nullptr;
    if (!desc) return fail(PFB_ERR_INVALID, "desc is NULL");
    if (desc->hbm_budget_bytes <= 0) return fail(PFB_ERR_INVALID, "hbm_budget_bytes must be > 0");
    if (desc->max_slots < 1 || desc->max_slots > 64) return fail(PFB_ERR_INVALID, "max_slots must be in [1, 64]");
    if (desc->timeout_ms < 1) return fail(PFB_ERR_INVALID, "timeout_ms must be >= 1");
    if (desc->queue_when_busy != 0 && desc->queue_when_busy != 1) return fail(PFB_ERR_INVALID, "queue_when_busy must be 0 or 1");
    int ndev = 0;
    PFB_CUDA_TRY(cudaGetDeviceCount(&ndev));
    int dev = desc->device;
    if (dev < 0) PFB_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= ndev) return fail(PFB_ERR_INVALID, "device ordinal out of range");
    Server *s = new (std::nothrow) Server();
    if (!s) return fail(PFB_ERR_OOM, "host allocation");
    s->desc = *desc;
    s->device = dev;
    parse_faults(*s);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
    const int npool = std::min(desc->max_slots, 16);
    for (int i = 0; i < npool; ++i) {
        cudaStream_t cs;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (auto p : s->pool) cudaStreamDestroy(p);
            cudaSetDevice(prev);
            delete s;
            return cuda_fail(e, "cudaStreamCreate");
        }
        s->pool.push_back(cs);
    }
    {
        pfb_status est = alloc_error_words(Server::kErrWords, &s->h_err, &s->d_err);
        if (est != PFB_OK) {
            for (auto p : s->pool) cudaStreamDestroy(p);
            cudaSetDevice(prev);
            delete s;
            return est;
        }
        for (int i = Server::kErrWords - 1; i >= 0; --i) s->free_err.push_back(i);
    }
    cudaSetDevice(prev);
    s->worker = std::thread(worker_loop, s);
    *out_server = reinterpret_cast<pfb_server_t>(s);
    return PFB_OK;
}

extern "C" pfb_status pfb_server_destroy(pfb_server_t server) {
    clear_error();
    if (!server) return PFB_OK;
    Server *s = reinterpret_cast<Server *>(server);
    pfb_status result = PFB_OK;
    {
        // bounded wait for queued and in-flight work
        std::unique_lock<std::mutex> lk(s->mu);
        const auto limit = Clock::now() + std::chrono::milliseconds((int64_t)s->desc.timeout_ms * 2 + 100);
        while ((!s->batches.empty() || !s->queue.empty()) && Clock::now() < limit) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(200));
            lk.lock();
        }
        if (!s->batches.empty() || !s->queue.empty()) result = fail(PFB_ERR_TIMEOUT, "work still in flight at destroy");
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (auto cs : s->pool) cudaStreamSynchronize(cs);
    for (auto &b : s->batches)
        if (b->done) cudaEventDestroy(b->done);
    for (auto e : s->free_events) cudaEventDestroy(e);
    for (auto &kv : s->streams) {
        cudaFree(kv.second->state[0]);
        cudaFree(kv.second->state[1]);
    }
    for (auto cs : s->pool) cudaStreamDestroy(cs);
    free_error_words(s->h_err);
    cudaSetDevice(prev);
    delete s;
    return result;
}

extern "C" pfb_status pfb_stream_open(pfb_server_t server, pfb_plan_t plan, int64_t *out_stream_id) {
    clear_error();
    if (!server || !plan || !out_stream_id) return fail(PFB_ERR_INVALID, "NULL argument");
    Server &s = *reinterpret_cast<Server *>(server);
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (p->device != s.device) return fail(PFB_ERR_INVALID, "plan is on another device");
    if (p->R > 1) return fail(PFB_ERR_UNSUPPORTED, "streams of oversampled plans (hop < P) are not served");
    const int64_t bytes = (int64_t)std::max(p->T - 1, 1) * p->P * p->esize;
    std::lock_guard<std::mutex> lk(s.mu);
    if (s.reserved + 2 * bytes > s.desc.hbm_budget_bytes) return fail(PFB_ERR_OOM, "stream state does not fit the budget");
    auto ps = std::make_unique<PStream>();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s.device);
    cudaError_t e = cudaMalloc(&ps->state[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&ps->state[1], bytes);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaFree(ps->state[0]);
        cudaFree(ps->state[1]);
        return fail(PFB_ERR_OOM, "stream state allocation");
    }
    ps->id = s.next_stream++;
    ps->plan = p;
    ps->state_bytes = 2 * bytes;
    s.reserved += ps->state_bytes;
    s.peak_reserved = std::max(s.peak_reserved, s.reserved);
    *out_stream_id = ps->id;
    s.streams[ps->id] = std::move(ps);
    return PFB_OK;
}

extern "C" pfb_status pfb_stream_close(pfb_server_t server, int64_t stream_id) {
    clear_error();
    if (!server) return fail(PFB_ERR_INVALID, "server is NULL");
    Server &s = *reinterpret_cast<Server *>(server);
    std::unique_lock<std::mutex> lk(s.mu);
    auto it = s.streams.find(stream_id);
    if (it == s.streams.end() || it->second->closing) return fail(PFB_ERR_INVALID, "unknown stream");
    PStream &ps = *it->second;
    ps.closing = true;
    const auto limit = Clock::now() + std::chrono::milliseconds((int64_t)s.desc.timeout_ms * 2 + 100);
    while (ps.outstanding > 0 && Clock::now() < limit) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(100));
        lk.lock();
    }
    if (ps.outstanding > 0) return fail(PFB_ERR_TIMEOUT, "stream still has work in flight");
    // wait until no in-flight request of this stream can still read the state
    bool busy = true;
    while (busy && Clock::now() < limit) {
        busy = false;
        for (auto &b : s.batches)
            for (Request *r : b->reqs)
                if (r->stream_id == stream_id && !r->released) busy = true;
        if (busy) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(100));
            lk.lock();
        }
    }
    if (busy) return fail(PFB_ERR_TIMEOUT, "stream state still in use");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s.device);
    if (ps.last_event) cudaEventSynchronize(ps.last_event);
    cudaFree(ps.state[0]);
    cudaFree(ps.state[1]);
    cudaSetDevice(prev);
    s.reserved -= ps.state_bytes;
    s.streams.erase(it);
    return PFB_OK;
}

static int64_t next_spectra_locked(const PStream &ps, int64_t n_samples) {
    const int64_t T = ps.plan->T;
    const int64_t st = std::min<int64_t>(T - 1, ps.frames_submitted);
    const int64_t S = st + n_samples / ps.plan->P - T + 1;
    return S > 0 ? S : 0;
}

extern "C" int64_t pfb_stream_next_spectra(pfb_server_t server, int64_t stream_id, int64_t n_samples) {
    if (!server || n_samples < 0) return -1;
    Server &s = *reinterpret_cast<Server *>(server);
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.streams.find(stream_id);
    if (it == s.streams.end()) return -1;
    return next_spectra_locked(*it->second, n_samples);
}

extern "C" pfb_status pfb_submit(pfb_server_t server, int64_t stream_id, const void *d_chunk, int64_t n_samples,
                                 void *d_out, int64_t out_cap_spectra, int64_t *out_ticket) {
    clear_error();
    if (!server || !out_ticket) return fail(PFB_ERR_INVALID, "NULL argument");
    *out_ticket = 0;
    Server &s = *reinterpret_cast<Server *>(server);
    const auto t0 = Clock::now();
    std::unique_lock<std::mutex> lk(s.mu);
    auto it = s.streams.find(stream_id);
    if (it == s.streams.end() || it->second->closing) return fail(PFB_ERR_INVALID, "unknown stream");
    PStream &ps = *it->second;
    const Plan &plan = *ps.plan;
    if (n_samples <= 0 || n_samples % plan.P != 0) return fail(PFB_ERR_INVALID, "chunk length must be a positive multiple of P");
    if (!d_chunk || (reinterpret_cast<uintptr_t>(d_chunk) & 15u)) return fail(PFB_ERR_INVALID, "chunk must be a 16-byte aligned device pointer");
    const int64_t S = next_spectra_locked(ps, n_samples);
    if (S > 0 && (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 15u)))
        return fail(PFB_ERR_INVALID, "output must be a 16-byte aligned device pointer");
    if (out_cap_spectra < S) return fail(PFB_ERR_INVALID, "out_cap_spectra smaller than the spectra produced");
    const int64_t bytes = n_samples * plan.esize + S * plan.P * (int64_t)sizeof(float2);
    if (bytes + ps.state_bytes > s.desc.hbm_budget_bytes) return fail(PFB_ERR_BUSY, "request larger than the budget");
    const bool fits = s.queue.empty() && s.inflight < s.desc.max_slots &&
                      s.reserved + bytes <= s.desc.hbm_budget_bytes;
    if (!fits && !s.desc.queue_when_busy) {
        s.n_rejected++;
        return fail(PFB_ERR_BUSY, "no slot or budget free");
    }
    auto r = std::make_unique<Request>();
    r->ticket = s.next_ticket++;
    r->stream_id = stream_id;
    r->d_chunk = d_chunk;
    r->d_out = d_out;
    r->n_samples = n_samples;
    r->S = S;
    r->bytes = bytes;
    r->t_submit = t0;
    ps.frames_submitted += n_samples / plan.P;
    ps.outstanding++;
    s.n_submitted++;
    Request *rp = r.get();
    *out_ticket = r->ticket;
    s.tickets[r->ticket] = std::move(r);
    s.queue.push_back(rp);
    lk.unlock();
    s.cv_work.notify_all();
    return PFB_OK;
}

extern "C" pfb_status pfb_poll(pfb_server_t server, int64_t ticket) {
    if (!server) return PFB_ERR_INVALID;
    Server &s = *reinterpret_cast<Server *>(server);
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.tickets.find(ticket);
    if (it == s.tickets.end()) return PFB_ERR_INVALID;
    return it->second->status;
}

extern "C" pfb_status pfb_submit_chunks(pfb_server_t server, int64_t stream_id, const void *d_chunks,
                                        int32_t n_chunks, int64_t samples_per_chunk, void *d_out,
                                        int64_t out_cap_spectra, int64_t *out_tickets) {
    clear_error();
    if (!server || !out_tickets) return fail(PFB_ERR_INVALID, "NULL argument");
    if (n_chunks < 1) return fail(PFB_ERR_INVALID, "n_chunks must be >= 1");
    for (int32_t i = 0; i < n_chunks; ++i) out_tickets[i] = 0;
    Server &s = *reinterpret_cast<Server *>(server);
    int64_t esize = 0, P = 0;
    {
        std::lock_guard<std::mutex> lk(s.mu);
        auto it = s.streams.find(stream_id);
        if (it == s.streams.end() || it->second->closing) return fail(PFB_ERR_INVALID, "unknown stream");
        esize = it->second->plan->esize;
        P = it->second->plan->P;
    }
    const char *in = static_cast<const char *>(d_chunks);
    float2 *out = static_cast<float2 *>(d_out);
    int64_t row = 0;
    for (int32_t i = 0; i < n_chunks; ++i) {
        const int64_t S = pfb_stream_next_spectra(server, stream_id, samples_per_chunk);
        if (S < 0) return fail(PFB_ERR_INVALID, "unknown stream");
        if (row + S > out_cap_spectra) return fail(PFB_ERR_INVALID, "out_cap_spectra smaller than the spectra produced");
        pfb_status st = pfb_submit(server, stream_id, in + (int64_t)i * samples_per_chunk * esize, samples_per_chunk,
                                   S > 0 ? static_cast<void *>(out + row * P) : nullptr, S, &out_tickets[i]);
        if (st != PFB_OK) return st;
        row += S;
    }
    return PFB_OK;
}

extern "C" pfb_status pfb_ticket_times(pfb_server_t server, int64_t ticket, double *t_submit_s, double *t_done_s) {
    clear_error();
    if (!server || !t_submit_s || !t_done_s) return fail(PFB_ERR_INVALID, "NULL argument");
    Server &s = *reinterpret_cast<Server *>(server);
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.tickets.find(ticket);
    if (it == s.tickets.end()) return fail(PFB_ERR_INVALID, "unknown ticket");
    const Request &r = *it->second;
    auto secs = [](Clock::time_point tp) { return std::chrono::duration<double>(tp.time_since_epoch()).count(); };
    *t_submit_s = secs(r.t_submit);
    *t_done_s = r.status == PFB_PENDING ? 0.0 : secs(r.t_done);
    return PFB_OK;
}

extern "C" pfb_status pfb_wait(pfb_server_t server, int64_t ticket, int32_t timeout_ms) {
    clear_error();
    if (!server) return fail(PFB_ERR_INVALID, "server is NULL");
    Server &s = *reinterpret_cast<Server *>(server);
    std::unique_lock<std::mutex> lk(s.mu);
    auto it = s.tickets.find(ticket);
    if (it == s.tickets.end()) return fail(PFB_ERR_INVALID, "unknown ticket");
    Request *r = it->second.get();
    const bool ok = s.cv_done.wait_for(lk, std::chrono::milliseconds(std::max(timeout_ms, 0)),
                                       [&] { return r->status != PFB_PENDING; });
    if (!ok) return fail(PFB_ERR_TIMEOUT, "wait timed out");
    return r->status;
}

extern "C" pfb_status pfb_server_get_stats(pfb_server_t server, pfb_server_stats *out) {
    clear_error();
    if (!server || !out) return fail(PFB_ERR_INVALID, "NULL argument");
    Server &s = *reinterpret_cast<Server *>(server);
    std::lock_guard<std::mutex> lk(s.mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s.n_submitted;
    out->completed = s.n_completed;
    out->failed = s.n_failed;
    out->rejected = s.n_rejected;
    out->queued_now = (int64_t)s.queue.size();
    out->in_flight_now = s.inflight;
    out->reserved_bytes_now = s.reserved;
    out->peak_reserved_bytes = s.peak_reserved;
    out->samples_completed = s.samples_completed;
    out->batches = s.n_batches;
    out->batched_requests = s.n_batched_requests;
    if (!s.latencies_us.empty()) {
        std::vector<double> v = s.latencies_us;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            size_t idx = (size_t)std::min<double>(v.size() - 1, std::floor(q * (v.size() - 1) + 0.5));
            return v[idx];
        };
        out->p50_latency_us = pct(0.50);
        out->p99_latency_us = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_latency_us = sum / v.size();
    }
    return PFB_OK;
}

// ---------------------------------------------------------------------------
// filter-state checkpoint: export / import of a stream's resident state
// ---------------------------------------------------------------------------
namespace pfb {

struct StateHeader {
    char magic[8];                 // "PFBSTATE"
    int32_t version, P, T, in_dtype, esize, reserved;
    int64_t frames_submitted;      // frames of all chunks the stream has taken
    int64_t state_frames;          // frames that follow the header (<= T - 1)
};
static_assert(sizeof(StateHeader) == 48, "state header layout");

// Wait (bounded by the server's timeout) until no submitted or in-flight work
// of the stream remains and its last batch has finished on the device.  Called
// with the lock held; returns with it held.
static pfb_status wait_stream_idle(Server &s, std::unique_lock<std::mutex> &lk, PStream &ps, int64_t stream_id) {
    const auto limit = Clock::now() + std::chrono::milliseconds((int64_t)s.desc.timeout_ms * 2 + 100);
    auto busy = [&] {
        if (ps.outstanding > 0) return true;
        for (auto &b : s.batches)
            for (Request *r : b->reqs)
                if (r->stream_id == stream_id && !r->released) return true;
        return false;
    };
    while (busy() && Clock::now() < limit) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(100));
        lk.lock();
    }
    if (busy()) return fail(PFB_ERR_TIMEOUT, "stream still has work in flight");
    if (ps.failed) return fail(PFB_ERR_INVALID, "an earlier chunk of the stream failed: its state is not defined");
    if (ps.last_event) {
        cudaError_t e = cudaEventSynchronize(ps.last_event);
        if (e != cudaSuccess) return cuda_fail(e, "stream's last batch");
    }
    return PFB_OK;
}

static int64_t state_blob_bytes(const PStream &ps) {
    return (int64_t)sizeof(StateHeader) + ps.state_frames * ps.plan->P * ps.plan->esize;
}

}  // namespace pfb

extern "C" int64_t pfb_stream_state_size(pfb_server_t server, int64_t stream_id) {
    if (!server) return -1;
    Server &s = *reinterpret_cast<Server *>(server);
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.streams.find(stream_id);
    if (it == s.streams.end()) return -1;
    // the size once the submitted chunks have run: the header and min(T - 1, frames) frames
    const PStream &ps = *it->second;
    const int64_t frames = std::min<int64_t>(ps.plan->T - 1, ps.frames_submitted);
    return (int64_t)sizeof(StateHeader) + frames * ps.plan->P * ps.plan->esize;
}

extern "C" pfb_status pfb_stream_state_export(pfb_server_t server, int64_t stream_id, void *host_buf, int64_t cap) {
    clear_error();
    if (!server || !host_buf) return fail(PFB_ERR_INVALID, "NULL argument");
    Server &s = *reinterpret_cast<Server *>(server);
    std::unique_lock<std::mutex> lk(s.mu);
    auto it = s.streams.find(stream_id);
    if (it == s.streams.end() || it->second->closing) return fail(PFB_ERR_INVALID, "unknown stream");
    PStream &ps = *it->second;
    pfb_status st = wait_stream_idle(s, lk, ps, stream_id);
    if (st != PFB_OK) return st;
    const int64_t need = state_blob_bytes(ps);
    if (cap < need) return fail(PFB_ERR_INVALID, "buffer smaller than pfb_stream_state_size()");
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "PFBSTATE", 8);
    h.version = 1;
    h.P = ps.plan->P;
    h.T = ps.plan->T;
    h.in_dtype = ps.plan->in_dtype;
    h.esize = ps.plan->esize;
    h.frames_submitted = ps.frames_submitted;
    h.state_frames = ps.state_frames;
    std::memcpy(host_buf, &h, sizeof(h));
    if (ps.state_frames > 0) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(s.device);
        cudaError_t e = cudaMemcpy(static_cast<char *>(host_buf) + sizeof(h), ps.state[ps.cur],
                                   (size_t)(need - (int64_t)sizeof(h)), cudaMemcpyDeviceToHost);
        cudaSetDevice(prev);
        if (e != cudaSuccess) return cuda_fail(e, "state export copy");
    }
    return PFB_OK;
}

extern "C" pfb_status pfb_stream_state_import(pfb_server_t server, int64_t stream_id, const void *host_buf,
                                              int64_t size) {
    clear_error();
    if (!server || !host_buf) return fail(PFB_ERR_INVALID, "NULL argument");
    if (size < (int64_t)sizeof(StateHeader)) return fail(PFB_ERR_INVALID, "state blob shorter than its header");
    StateHeader h;
    std::memcpy(&h, host_buf, sizeof(h));
    if (std::memcmp(h.magic, "PFBSTATE", 8) != 0 || h.version != 1) return fail(PFB_ERR_INVALID, "not a state blob");
    Server &s = *reinterpret_cast<Server *>(server);
    std::unique_lock<std::mutex> lk(s.mu);
    auto it = s.streams.find(stream_id);
    if (it == s.streams.end() || it->second->closing) return fail(PFB_ERR_INVALID, "unknown stream");
    PStream &ps = *it->second;
    const Plan &plan = *ps.plan;
    if (h.P != plan.P || h.T != plan.T || h.in_dtype != plan.in_dtype || h.esize != plan.esize)
        return fail(PFB_ERR_INVALID, "state blob was exported from a stream of another P, T or dtype");
    if (h.frames_submitted < 0 || h.state_frames != std::min<int64_t>(plan.T - 1, h.frames_submitted))
        return fail(PFB_ERR_INVALID, "inconsistent state blob");
    const int64_t bytes = h.state_frames * plan.P * plan.esize;
    if (size < (int64_t)sizeof(h) + bytes) return fail(PFB_ERR_INVALID, "state blob truncated");
    pfb_status st = wait_stream_idle(s, lk, ps, stream_id);
    if (st != PFB_OK) return st;
    if (bytes > 0) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(s.device);
        cudaError_t e = cudaMemcpy(ps.state[ps.cur], static_cast<const char *>(host_buf) + sizeof(h), (size_t)bytes,
                                   cudaMemcpyHostToDevice);
        cudaSetDevice(prev);
        if (e != cudaSuccess) return cuda_fail(e, "state import copy");
    }
    ps.state_frames = h.state_frames;
    ps.frames_submitted = h.frames_submitted;
    return PFB_OK;
}
