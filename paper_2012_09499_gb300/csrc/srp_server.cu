// Serving engine: frame blocks from many arrays (one resident plan per
// array) are mapped as they arrive, by continuous batching.
//
//  - A worker thread forms iterations: every stream's queued requests, in
//    arrival order and up to the plan's max_frames, become one group of
//    consecutive frames; all groups of an iteration go to the GPU together
//    (one srp_map_batch graph launch over the tensor-core plans, srp_map for
//    the others) with their input copies before and result copies after.
//  - Up to max_inflight iterations are on the GPU at once, each on its own
//    CUDA stream with its own batch object, so requests that arrive while
//    others run are admitted into the next iteration as soon as a slot and
//    memory free up, and its copies and kernels overlap the running ones.
//  - HBM admission: every group's device working set (inputs, maps, argmax,
//    peak) is carved from one device arena of the budgeted size; a group
//    that does not fit waits for earlier ones to finish.  A request that
//    could never fit is refused at submission.
//  - Inputs are copied at submission into pinned staging (so the caller's
//    buffer is free at once); results return through pinned staging into
//    the caller's buffers, and each completion carries its submission,
//    start and completion times for latency statistics.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "srp_internal.h"

namespace srp {
namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over [0, size): offsets and sizes are multiples of kAlign.
class Arena {
  public:
    void init(size_t size) {
        size_ = size;
        free_.clear();
        if (size > 0) free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(size_t n, size_t *off) {
        n = align_up(std::max<size_t>(n, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n;
            const size_t start = it->first + n;
            free_.erase(it);
            if (rest > 0) free_[start] = rest;
            used_ += n;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = align_up(std::max<size_t>(n, 1));
        used_ -= n;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

struct Request {
    uint64_t id = 0, tag = 0;
    int stream = 0, L = 0;
    int32_t *h_argmax = nullptr;
    float *h_peak = nullptr;
    float *h_maps = nullptr;
    size_t pin_off = 0, pin_bytes = 0;  // pinned: input, then argmax and peak
    double t_submit = 0.0, t_deadline = 0.0, t_start = 0.0;
};

struct Group {  // one stream's requests in one iteration
    int stream = 0, L = 0;
    std::vector<Request> reqs;
    size_t dev_off = 0, dev_bytes = 0;
    char *d_in = nullptr;
    float *d_maps = nullptr;
    int32_t *d_argmax = nullptr;
    float *d_peak = nullptr;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t gpu_start = nullptr, gpu_end = nullptr;  // timed: the iteration's GPU interval
    srp_batch batch = nullptr;
    bool busy = false;
    std::vector<Group> groups;
    double t_start = 0.0;
    int64_t seq = 0;  // iteration number
};

struct Interval {  // GPU interval of a retired iteration
    int64_t seq = 0;
    double t0 = 0.0, t1 = 0.0;
    bool counted = false;
};
constexpr size_t kHistory = 16;  // retired iterations kept for the overlap count

struct StreamInfo {
    srp_plan_s *plan = nullptr;
    int batch_index = -1;   // index among the batched plans, or -1 (own srp_map call)
    size_t in_frame_bytes = 0;
    int64_t J = 0;
    int max_frames = 0;
    int solo_slot = -1;     // slot using this plan's own scratch, or -1
    std::deque<Request> queue;
};

}  // namespace
}  // namespace srp

using namespace srp;

struct srp_server_s {
    int device = 0;
    srp_server_desc desc{};
    std::vector<StreamInfo> streams;
    std::vector<srp_handle> batched;  // plans of the batch, in batch order
    std::vector<Slot> slots;
    char *d_arena = nullptr;
    Arena dev;
    char *h_pinned = nullptr;
    Arena pin;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<srp_completion> done;
    std::thread worker;
    bool stop = false;
    bool hold = false;  // srp_server_hold: queue requests, form no iteration
    std::chrono::steady_clock::time_point t0;
    uint64_t next_id = 1;
    int rr = 0;  // round-robin start of iteration forming
    srp_server_stats stats{};
    std::string worker_error;
    cudaEvent_t gpu_ref = nullptr;  // device time origin of the iteration intervals
    std::deque<Interval> history;   // the last kHistory retired iterations

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
            .count();
    }
};

namespace srp {
namespace {

size_t group_bytes(const StreamInfo &si, int L) {
    return align_up(si.in_frame_bytes * L) + align_up(sizeof(float) * (size_t)L * si.J) +
           2 * align_up(sizeof(int32_t) * L);
}

void server_release(srp_server_s *s) {
    for (Slot &sl : s->slots) {
        if (sl.batch) srp_batch_destroy(sl.batch);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.gpu_start) cudaEventDestroy(sl.gpu_start);
        if (sl.gpu_end) cudaEventDestroy(sl.gpu_end);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->gpu_ref) cudaEventDestroy(s->gpu_ref);
    cudaFree(s->d_arena);
    cudaFreeHost(s->h_pinned);
}

// Iteration of a completed request (all zero when it never ran).
struct IterInfo {
    int64_t seq = 0;
    int32_t streams = 0, frames = 0;
    double t_gpu0 = 0.0, t_gpu1 = 0.0;
};

void complete(srp_server_s *s, const Request &r, int status, double t_done,
              const IterInfo &it = IterInfo()) {
    srp_completion c;
    memset(&c, 0, sizeof c);
    c.request_id = r.id;
    c.tag = r.tag;
    c.stream = r.stream;
    c.L = r.L;
    c.status = status;
    c.t_submit_ms = r.t_submit;
    c.t_start_ms = r.t_start;
    c.t_done_ms = t_done;
    c.iteration = it.seq;
    c.iteration_streams = it.streams;
    c.iteration_frames = it.frames;
    c.t_gpu_start_ms = it.t_gpu0;
    c.t_gpu_end_ms = it.t_gpu1;
    s->done.push_back(c);
    if (status == SRP_OK) {
        s->stats.completed += 1;
        s->stats.frames_completed += r.L;
    } else if (status == SRP_ERR_TIMEOUT) {
        s->stats.timed_out += 1;
    } else {
        s->stats.failed += 1;
    }
}

// Retire finished iterations: deliver results, free memory.  Lock held.
void retire(srp_server_s *s) {
    for (size_t k = 0; k < s->slots.size(); ++k) {
        Slot &sl = s->slots[k];
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        const double t = s->now_ms();
        const int status = q == cudaSuccess ? SRP_OK : SRP_ERR_CUDA;
        if (q != cudaSuccess) s->worker_error = cudaGetErrorString(q);
        IterInfo it;
        it.seq = sl.seq;
        it.streams = (int32_t)sl.groups.size();
        for (const Group &g : sl.groups) it.frames += g.L;
        if (status == SRP_OK) {
            float a = 0.0f, b = 0.0f;
            if (cudaEventElapsedTime(&a, s->gpu_ref, sl.gpu_start) == cudaSuccess &&
                cudaEventElapsedTime(&b, s->gpu_ref, sl.gpu_end) == cudaSuccess) {
                it.t_gpu0 = a;
                it.t_gpu1 = b;
                // count this iteration (and an earlier one) once each if their
                // GPU intervals intersect
                bool mine = false;
                for (Interval &h : s->history)
                    if (h.t0 < it.t_gpu1 && it.t_gpu0 < h.t1) {
                        mine = true;
                        if (!h.counted) {
                            h.counted = true;
                            s->stats.overlapped_iterations += 1;
                        }
                    }
                if (mine) s->stats.overlapped_iterations += 1;
                Interval iv;
                iv.seq = it.seq;
                iv.t0 = it.t_gpu0;
                iv.t1 = it.t_gpu1;
                iv.counted = mine;
                s->history.push_back(iv);
                if (s->history.size() > kHistory) s->history.pop_front();
            }
        }
        for (Group &g : sl.groups) {
            for (Request &r : g.reqs) {
                if (status == SRP_OK) {
                    const char *res = s->h_pinned + r.pin_off + align_up(s->streams[r.stream].in_frame_bytes * r.L);
                    memcpy(r.h_argmax, res, sizeof(int32_t) * r.L);
                    if (r.h_peak != nullptr)
                        memcpy(r.h_peak, res + align_up(sizeof(int32_t) * r.L), sizeof(float) * r.L);
                }
                complete(s, r, status, t, it);
                s->pin.release(r.pin_off, r.pin_bytes);
            }
            s->dev.release(g.dev_off, g.dev_bytes);
            if (s->streams[g.stream].solo_slot == (int)k) s->streams[g.stream].solo_slot = -1;
        }
        sl.groups.clear();
        sl.busy = false;
        s->cv_done.notify_all();
    }
}

// Take queued requests into groups for slot k.  Lock held.  Returns false
// if nothing was taken.
bool form(srp_server_s *s, int k) {
    Slot &sl = s->slots[k];
    const double t = s->now_ms();
    const int n = (int)s->streams.size();
    for (int j = 0; j < n; ++j) {
        const int si_idx = (s->rr + j) % n;
        StreamInfo &si = s->streams[si_idx];
        // requests whose deadline passed before they could start
        while (!si.queue.empty() && si.queue.front().t_deadline > 0.0 &&
               si.queue.front().t_deadline < t) {
            complete(s, si.queue.front(), SRP_ERR_TIMEOUT, t);
            s->pin.release(si.queue.front().pin_off, si.queue.front().pin_bytes);
            si.queue.pop_front();
        }
        if (si.queue.empty()) continue;
        if (si.batch_index < 0 && si.solo_slot >= 0) continue;  // its scratch is in use
        int L = 0;
        size_t cnt = 0;
        while (cnt < si.queue.size() && L + si.queue[cnt].L <= si.max_frames &&
               (si.queue[cnt].t_deadline <= 0.0 || si.queue[cnt].t_deadline >= t)) {
            L += si.queue[cnt].L;
            ++cnt;
        }
        if (cnt == 0) continue;
        // admission: shrink the group until its working set fits the arena
        size_t off = 0, bytes = 0;
        bool ok = false;
        while (cnt > 0) {
            bytes = group_bytes(si, L);
            if (s->dev.alloc(bytes, &off)) {
                ok = true;
                break;
            }
            --cnt;
            L -= si.queue[cnt].L;
        }
        if (!ok) {
            s->stats.admission_waits += 1;
            continue;
        }
        Group g;
        g.stream = si_idx;
        g.L = L;
        g.dev_off = off;
        g.dev_bytes = bytes;
        char *base = s->d_arena + off;
        g.d_in = base;
        base += align_up(si.in_frame_bytes * L);
        g.d_maps = reinterpret_cast<float *>(base);
        base += align_up(sizeof(float) * (size_t)L * si.J);
        g.d_argmax = reinterpret_cast<int32_t *>(base);
        base += align_up(sizeof(int32_t) * L);
        g.d_peak = reinterpret_cast<float *>(base);
        for (size_t c = 0; c < cnt; ++c) {
            Request r = si.queue.front();
            si.queue.pop_front();
            r.t_start = t;
            g.reqs.push_back(r);
        }
        if (si.batch_index < 0) si.solo_slot = k;
        sl.groups.push_back(std::move(g));
    }
    s->rr = (s->rr + 1) % std::max(1, n);
    return !sl.groups.empty();
}

// Enqueue copies and kernels of slot k's groups.  Lock not held.
srp_status launch(srp_server_s *s, int k) {
    Slot &sl = s->slots[k];
    cudaStream_t st = sl.stream;
    const int nb = (int)s->batched.size();
    std::vector<const void *> in(nb, nullptr);
    std::vector<int32_t> Ls(nb, 0);
    std::vector<float *> maps(nb, nullptr), peaks(nb, nullptr);
    std::vector<int32_t *> ams(nb, nullptr);
    bool any_batch = false;
    int launches = 0;
    SRP_CUDA(cudaEventRecord(sl.gpu_start, st), "record iteration start");
    for (Group &g : sl.groups) {
        const StreamInfo &si = s->streams[g.stream];
        int f = 0;
        for (const Request &r : g.reqs) {
            SRP_CUDA(cudaMemcpyAsync(g.d_in + si.in_frame_bytes * f, s->h_pinned + r.pin_off,
                                     si.in_frame_bytes * r.L, cudaMemcpyHostToDevice, st),
                     "copy request input");
            f += r.L;
        }
        if (si.batch_index >= 0) {
            in[si.batch_index] = g.d_in;
            Ls[si.batch_index] = g.L;
            maps[si.batch_index] = g.d_maps;
            ams[si.batch_index] = g.d_argmax;
            peaks[si.batch_index] = g.d_peak;
            any_batch = true;
        } else {
            srp_status r = srp_map(si.plan, g.d_in, g.L, g.d_maps, g.d_argmax, g.d_peak,
                                   reinterpret_cast<srp_stream_t>(st));
            if (r != SRP_OK) return r;
            launches += si.plan->last_launches;
        }
    }
    if (any_batch) {
        srp_status r = srp_map_batch(sl.batch, in.data(), Ls.data(), maps.data(), ams.data(),
                                     peaks.data(), reinterpret_cast<srp_stream_t>(st));
        if (r != SRP_OK) return r;
        launches += 3;
    }
    for (Group &g : sl.groups) {
        const StreamInfo &si = s->streams[g.stream];
        int f = 0;
        for (const Request &r : g.reqs) {
            char *res = s->h_pinned + r.pin_off + align_up(si.in_frame_bytes * r.L);
            SRP_CUDA(cudaMemcpyAsync(res, g.d_argmax + f, sizeof(int32_t) * r.L,
                                     cudaMemcpyDeviceToHost, st), "copy argmax");
            SRP_CUDA(cudaMemcpyAsync(res + align_up(sizeof(int32_t) * r.L), g.d_peak + f,
                                     sizeof(float) * r.L, cudaMemcpyDeviceToHost, st),
                     "copy peak");
            if (r.h_maps != nullptr)
                SRP_CUDA(cudaMemcpyAsync(r.h_maps, g.d_maps + (size_t)f * si.J,
                                         sizeof(float) * (size_t)r.L * si.J,
                                         cudaMemcpyDeviceToHost, st), "copy maps");
            f += r.L;
        }
    }
    SRP_CUDA(cudaEventRecord(sl.gpu_end, st), "record iteration end");
    SRP_CUDA(cudaEventRecord(sl.done, st), "record iteration event");
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.kernel_launches += launches;
    return SRP_OK;
}

void worker_main(srp_server_s *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        retire(s);
        bool busy = false, pending = false;
        for (const Slot &sl : s->slots) busy |= sl.busy;
        for (const StreamInfo &si : s->streams) pending |= !si.queue.empty();
        if (s->stop && !busy && !pending) break;
        int k = -1;
        for (size_t j = 0; j < s->slots.size(); ++j)
            if (!s->slots[j].busy) {
                k = (int)j;
                break;
            }
        if (k >= 0 && pending && !(s->hold && !s->stop) && form(s, k)) {
            Slot &sl = s->slots[k];
            sl.busy = true;
            sl.t_start = s->now_ms();
            s->stats.iterations += 1;
            sl.seq = s->stats.iterations;
            s->stats.max_iteration_streams =
                std::max(s->stats.max_iteration_streams, (int32_t)sl.groups.size());
            lk.unlock();
            srp_status st = launch(s, k);
            lk.lock();
            if (st != SRP_OK) {
                // nothing of this iteration may still run: wait for its stream,
                // then fail its requests and free their memory
                lk.unlock();
                cudaStreamSynchronize(sl.stream);
                lk.lock();
                s->worker_error = srp_last_error_message();
                const double t = s->now_ms();
                for (Group &g : sl.groups) {
                    for (Request &r : g.reqs) {
                        complete(s, r, st, t);
                        s->pin.release(r.pin_off, r.pin_bytes);
                    }
                    s->dev.release(g.dev_off, g.dev_bytes);
                    if (s->streams[g.stream].solo_slot == k) s->streams[g.stream].solo_slot = -1;
                }
                sl.groups.clear();
                sl.busy = false;
                s->cv_done.notify_all();
            }
            continue;
        }
        // nothing to start: sleep until a submission or a short poll interval
        s->cv_work.wait_for(lk, std::chrono::microseconds(busy ? 20 : 2000));
    }
}

}  // namespace
}  // namespace srp

extern "C" {

srp_status srp_server_create(const srp_handle *plans, int32_t n, const srp_server_desc *d,
                             srp_server *out) {
    if (out == nullptr || plans == nullptr || n < 1 || d == nullptr)
        return fail(SRP_ERR_INVALID_ARG, "plans, n >= 1, desc and out are required");
    if (d->device_budget_bytes == 0 || d->host_budget_bytes == 0)
        return fail(SRP_ERR_INVALID_ARG, "device and host budgets must be > 0");
    if (d->max_inflight < 1 || d->max_inflight > 8)
        return fail(SRP_ERR_INVALID_ARG, "max_inflight must be in [1, 8]");
    for (int i = 0; i < n; ++i)
        if (plans[i] == nullptr) return fail(SRP_ERR_INVALID_ARG, "plan handle is NULL");
    for (int i = 1; i < n; ++i)
        if (plans[i]->device != plans[0]->device)
            return fail(SRP_ERR_INVALID_ARG, "plans on different devices");
    DeviceGuard g(plans[0]->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plans' device");
    srp_server_s *s = new (std::nothrow) srp_server_s();
    if (s == nullptr) return fail(SRP_ERR_OOM, "host allocation failed");
    auto bail = [&](srp_status st) {
        server_release(s);
        delete s;
        return st;
    };
    s->device = plans[0]->device;
    s->desc = *d;
    s->t0 = std::chrono::steady_clock::now();
    // plans batched together: tensor-core plans of the first such plan's mode
    // and precision (unless batching is off); the rest map on their own
    const srp_plan_s *lead = nullptr;
    for (int i = 0; i < n; ++i)
        if (plans[i]->lay.tc && !d->no_batching) {
            lead = plans[i];
            break;
        }
    s->streams.resize(n);
    for (int i = 0; i < n; ++i) {
        StreamInfo &si = s->streams[i];
        srp_plan_s *p = plans[i];
        si.plan = p;
        const int rows = p->input_kind == SRP_IN_STFT ? p->lay.M : p->lay.Q;
        si.in_frame_bytes = sizeof(float) * 2 * (size_t)rows * p->lay.Kb;
        si.J = p->lay.J;
        si.max_frames = p->lay.L_max;
        if (lead != nullptr && p->lay.tc && p->mode == lead->mode &&
            p->precision == lead->precision) {
            si.batch_index = (int)s->batched.size();
            s->batched.push_back(p);
        }
    }
    cudaError_t e;
    if ((e = cudaMalloc(&s->d_arena, d->device_budget_bytes)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMalloc server arena"));
    s->dev.init(d->device_budget_bytes / kAlign * kAlign);
    if ((e = cudaMallocHost(&s->h_pinned, d->host_budget_bytes)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMallocHost server staging"));
    s->pin.init(d->host_budget_bytes / kAlign * kAlign);
    s->slots.resize(d->max_inflight);
    for (Slot &sl : s->slots) {
        if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreate(&sl.gpu_start)) != cudaSuccess ||
            (e = cudaEventCreate(&sl.gpu_end)) != cudaSuccess)
            return bail(cuda_fail(e, "server stream"));
        if (!s->batched.empty()) {
            srp_status st = srp_batch_create(s->batched.data(), (int32_t)s->batched.size(),
                                             nullptr, &sl.batch);
            if (st != SRP_OK) return bail(st);
        }
    }
    // the origin of the iterations' GPU intervals, complete before any iteration
    if ((e = cudaEventCreate(&s->gpu_ref)) != cudaSuccess ||
        (e = cudaEventRecord(s->gpu_ref, s->slots[0].stream)) != cudaSuccess ||
        (e = cudaEventSynchronize(s->gpu_ref)) != cudaSuccess)
        return bail(cuda_fail(e, "server time origin"));
    s->stats.device_budget_bytes = s->dev.size();
    s->stats.batched_streams = (int32_t)s->batched.size();
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        return bail(fail(SRP_ERR_OOM, "cannot start the server thread"));
    }
    *out = s;
    return SRP_OK;
}

srp_status srp_server_submit(srp_server s, int32_t stream, const void *h_in, int32_t L,
                             int32_t *h_argmax, float *h_peak, float *h_maps, uint64_t tag,
                             double deadline_ms, uint64_t *request_id) {
    if (s == nullptr) return fail(SRP_ERR_INVALID_ARG, "server is NULL");
    if (stream < 0 || stream >= (int32_t)s->streams.size())
        return fail(SRP_ERR_INVALID_ARG, "stream out of range");
    StreamInfo &si = s->streams[stream];
    if (L < 1 || L > si.max_frames) return fail(SRP_ERR_INVALID_ARG, "L out of [1, max_frames]");
    if (h_in == nullptr || h_argmax == nullptr)
        return fail(SRP_ERR_INVALID_ARG, "h_in and h_argmax must be non-NULL");
    const size_t need_dev = group_bytes(si, L);
    const size_t pin_bytes = align_up(si.in_frame_bytes * L) + 2 * align_up(sizeof(int32_t) * L);
    std::unique_lock<std::mutex> lk(s->mu);
    if (need_dev > s->dev.size() || pin_bytes > s->pin.size()) {
        s->stats.rejected += 1;
        return fail(SRP_ERR_OOM, "request exceeds the server's memory budget");
    }
    size_t off = 0;
    if (!s->pin.alloc(pin_bytes, &off)) {
        s->stats.rejected += 1;
        return fail(SRP_ERR_OOM, "host staging full (too many requests queued)");
    }
    Request r;
    r.id = s->next_id++;
    r.tag = tag;
    r.stream = stream;
    r.L = L;
    r.h_argmax = h_argmax;
    r.h_peak = h_peak;
    r.h_maps = h_maps;
    r.pin_off = off;
    r.pin_bytes = pin_bytes;
    r.t_submit = s->now_ms();
    r.t_deadline = deadline_ms > 0.0 ? r.t_submit + deadline_ms : 0.0;
    lk.unlock();
    memcpy(s->h_pinned + off, h_in, si.in_frame_bytes * L);  // the region is this request's
    lk.lock();
    si.queue.push_back(r);
    s->stats.submitted += 1;
    if (request_id != nullptr) *request_id = r.id;
    lk.unlock();
    s->cv_work.notify_one();
    return SRP_OK;
}

srp_status srp_server_poll(srp_server s, srp_completion *out, int32_t max, int32_t *n_out,
                           int32_t wait_ms) {
    if (s == nullptr || n_out == nullptr || (max > 0 && out == nullptr) || max < 0)
        return fail(SRP_ERR_INVALID_ARG, "bad argument");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms),
                            [&] { return !s->done.empty(); });
    int k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = k;
    return SRP_OK;
}

srp_status srp_server_hold(srp_server s, int32_t hold) {
    if (s == nullptr) return fail(SRP_ERR_INVALID_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->hold = hold != 0;
    }
    s->cv_work.notify_all();
    return SRP_OK;
}

srp_status srp_server_get_stats(srp_server s, srp_server_stats *st) {
    if (s == nullptr || st == nullptr) return fail(SRP_ERR_INVALID_ARG, "bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->stats;
    st->device_bytes_in_use = s->dev.used();
    st->device_bytes_peak = s->dev.peak();
    int64_t q = 0;
    for (const StreamInfo &si : s->streams) q += (int64_t)si.queue.size();
    st->queued = q;
    return SRP_OK;
}

srp_status srp_server_destroy(srp_server s) {
    if (s == nullptr) return SRP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    {
        DeviceGuard g(s->device);
        server_release(s);
    }
    delete s;
    return SRP_OK;
}

}  // extern "C"
