// flic_serve.cu — the serving loop: continuous batching of frames from several sensors.
//
// Requests (range images or xyz clouds in host memory) are queued by flic_server_submit.
// One dispatcher thread admits them into free frame slots — device memory reserved per
// sensor at creation, so admission is by device memory — and, whenever one of its
// streams ("lanes") is idle, launches everything admitted as one batch on that lane:
// host-to-device copies, the projection of all clouds of the batch (one launch each to
// clear the keys, project the points and decode the range images, every cloud on its
// slot's own handle, so concurrent projections never share scratch), one flic_label_batch
// for all frames, one scatter launch for all clouds, device-to-host copies, and a host
// callback that time-stamps completion.  While one lane's batch runs, requests that arrive are
// admitted and launched on the next lane, so batches overlap on the device.  Each frame's
// results equal the single-frame calls: the kernels decide every pixel and point the same
// way whatever else shares the launch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "flic.h"
#include "flic_internal.h"

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    static const clk::time_point t0 = clk::now();
    return std::chrono::duration<double>(clk::now() - t0).count();
}

struct Slot {
    int sensor = 0;
    flic_handle h = nullptr;  // this slot's tables and projection scratch
    float* d_range = nullptr;
    int32_t* d_labels = nullptr;
    float* d_xyz = nullptr;
    int32_t* d_pix = nullptr;
    int32_t* d_plab = nullptr;
};

struct Request {
    int sensor = 0;
    int kind = 0;
    const void* in = nullptr;
    int64_t n = 0;
    int32_t* out = nullptr;
    uint64_t tag = 0;
    double t_submit = 0.0;
};

struct Flight {  // one batch in flight on one lane
    std::condition_variable* cv = nullptr;  // the server's, woken at completion
    std::vector<int> slots;
    std::vector<Request> reqs;
    double t_launch = 0.0;
    std::atomic<double> t_done{0.0};
    std::atomic<int> done{0};
    int status = FLIC_OK;
};

struct Lane {
    cudaStream_t stream = nullptr;
    flic_batch batch = nullptr;
    // small batches (too few batch-sized strips to give every SM one): 2048-pixel strips,
    // so that more blocks share the frames and the batch finishes sooner
    flic_batch batch_small = nullptr;
    bool busy = false;
    Flight f;
    std::vector<flic::ProjBatch> proj;  // the batch's projection items (launch parameters)
};

struct Sensor {
    int rows = 0, cols = 0;
    int64_t max_points = 0;
    std::vector<int> free_slots;
};

void CUDART_CB on_batch_done(void* p) {
    Flight* f = static_cast<Flight*>(p);
    f->t_done.store(now_s());
    f->done.store(1);
    f->cv->notify_all();
}

}  // namespace

struct flic_server_ctx {
    std::vector<Sensor> sensors;
    std::vector<Slot> slots;
    std::deque<Lane> lanes;  // not movable (atomics): built in place
    int max_batch = 0;
    size_t small_px = 0;  // batches of fewer pixels use the lane's small-strip object
    int max_queue = 0;
    int64_t slot_bytes = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::vector<flic_completion> completions;
    std::thread dispatcher;
    std::atomic<bool> stop{false};
    std::atomic<bool> hold{false};  // admission paused by flic_server_hold
    int64_t submitted = 0, rejected = 0, completed = 0, batches = 0, largest = 0;
    int in_flight = 0;
    int device = 0;
};

namespace {

void free_server(flic_server_ctx* s) {
    for (Slot& sl : s->slots) {
        flic_destroy(sl.h);
        cudaFree(sl.d_range);
        cudaFree(sl.d_labels);
        cudaFree(sl.d_xyz);
        cudaFree(sl.d_pix);
        cudaFree(sl.d_plab);
    }
    for (Lane& ln : s->lanes) {
        if (ln.batch) flic_batch_destroy(ln.batch);
        if (ln.batch_small) flic_batch_destroy(ln.batch_small);
        if (ln.stream) cudaStreamDestroy(ln.stream);
    }
    delete s;
}

flic_status srv_fail(flic_status st, const char* msg) {
    flic::set_last_error(msg);
    return st;
}

void dispatch_loop(flic_server_ctx* s);

}  // namespace

extern "C" double flic_server_clock(void) { return now_s(); }

extern "C" flic_status flic_server_create(const flic_handle* sensors, int32_t nsensors,
                                          const int64_t* max_points, int32_t nstreams,
                                          int32_t max_batch, int64_t mem_budget,
                                          int32_t max_queue, flic_server* out) {
    if (!out) return srv_fail(FLIC_ERR_INVALID, "flic_server_create: out is NULL");
    *out = nullptr;
    if (!sensors || nsensors < 1 || nsensors > 64 || nstreams < 1 || nstreams > 8 ||
        max_batch < 1 || max_batch > 4096 || mem_budget < 0 || max_queue < 1)
        return srv_fail(FLIC_ERR_INVALID, "flic_server_create: bad argument");
    flic_server_ctx* s = new flic_server_ctx();
    s->max_batch = max_batch;
    s->max_queue = max_queue;
    cudaGetDevice(&s->device);
    s->sensors.resize(nsensors);
    // bytes of one slot per sensor, and how many slots of each fit the budget
    std::vector<int64_t> per(nsensors);
    int64_t round = 0;
    for (int i = 0; i < nsensors; ++i) {
        if (!sensors[i]) {
            free_server(s);
            return srv_fail(FLIC_ERR_INVALID, "flic_server_create: NULL sensor handle");
        }
        int64_t mp = max_points ? max_points[i] : 0;
        if (mp < 0 || mp >= ((int64_t)1 << 31)) {
            free_server(s);
            return srv_fail(FLIC_ERR_INVALID, "flic_server_create: bad max_points");
        }
        s->sensors[i].max_points = mp;
        int rows = 0, cols = 0;
        flic_handle probe = nullptr;
        flic_status st = flic::clone_handle(sensors[i], &probe, &rows, &cols);
        if (st != FLIC_OK) {
            free_server(s);
            return st;
        }
        flic_destroy(probe);
        s->sensors[i].rows = rows;
        s->sensors[i].cols = cols;
        per[i] = (int64_t)rows * cols * 8 + mp * 20;
        round += per[i];
    }
    const int64_t nper = std::max<int64_t>(1, round > 0 ? mem_budget / round : 1);
    for (int i = 0; i < nsensors; ++i) {
        for (int64_t k = 0; k < nper; ++k) {
            Slot sl;
            sl.sensor = i;
            int rows = 0, cols = 0;
            flic_status st = flic::clone_handle(sensors[i], &sl.h, &rows, &cols);
            cudaError_t e = cudaSuccess;
            const size_t npix = (size_t)rows * cols;
            const size_t mp = (size_t)s->sensors[i].max_points;
            if (st == FLIC_OK &&
                ((e = cudaMalloc((void**)&sl.d_range, npix * 4)) != cudaSuccess ||
                 (e = cudaMalloc((void**)&sl.d_labels, npix * 4)) != cudaSuccess ||
                 (mp && (e = cudaMalloc((void**)&sl.d_xyz, mp * 12)) != cudaSuccess) ||
                 (mp && (e = cudaMalloc((void**)&sl.d_pix, mp * 4)) != cudaSuccess) ||
                 (mp && (e = cudaMalloc((void**)&sl.d_plab, mp * 4)) != cudaSuccess)))
                st = e == cudaErrorMemoryAllocation ? FLIC_ERR_OOM : FLIC_ERR_CUDA;
            s->slots.push_back(sl);
            if (st != FLIC_OK) {
                cudaGetLastError();
                free_server(s);
                return srv_fail(st, "flic_server_create: slot allocation failed");
            }
            s->sensors[i].free_slots.push_back((int)s->slots.size() - 1);
            s->slot_bytes += per[i];
        }
    }
    for (int i = 0; i < nstreams; ++i) s->lanes.emplace_back();
    for (Lane& ln : s->lanes) {
        cudaError_t e = cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking);
        flic_status st = e == cudaSuccess ? flic_batch_create(max_batch, &ln.batch) : FLIC_ERR_CUDA;
        if (st == FLIC_OK) st = flic_batch_create(max_batch, &ln.batch_small);
        if (st == FLIC_OK) st = flic_batch_set_tuning(ln.batch_small, 2048, 0, 0, 0);
        if (st != FLIC_OK) {
            free_server(s);
            return srv_fail(st, "flic_server_create: stream or batch object failed");
        }
    }
    {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        s->small_px = (size_t)std::max(nsm, 1) * 16384;  // one batch-sized strip per SM
    }
    // one launch shape per batch object whatever the sensor mix, captured now: every batch
    // object reserves the shared memory of its largest sensor and labels one slot of each
    // sensor once (zeroed readings), so that no graph is captured while frames are served
    {
        std::vector<flic_handle> hs;
        std::vector<const float*> rs;
        std::vector<int32_t*> ls;
        for (const Sensor& sn : s->sensors) {
            const Slot& sl = s->slots[sn.free_slots.front()];
            hs.push_back(sl.h);
            rs.push_back(sl.d_range);
            ls.push_back(sl.d_labels);
            cudaMemset(sl.d_range, 0, (size_t)sn.rows * sn.cols * 4);
        }
        const int n = (int)hs.size();
        flic_status st = FLIC_OK;
        for (Lane& ln : s->lanes) {
            for (flic_batch b : {ln.batch, ln.batch_small}) {
                if (st == FLIC_OK) st = flic::batch_reserve_smem(b, hs.data(), n);
                if (st == FLIC_OK)
                    st = flic_label_batch(b, hs.data(), rs.data(), ls.data(), n, ln.stream);
            }
            if (st == FLIC_OK && cudaStreamSynchronize(ln.stream) != cudaSuccess) st = FLIC_ERR_CUDA;
        }
        if (st != FLIC_OK) {
            free_server(s);
            return srv_fail(st, "flic_server_create: warm-up launch failed");
        }
    }
    s->dispatcher = std::thread(dispatch_loop, s);
    *out = s;
    return FLIC_OK;
}

namespace {

// Enqueue one batch on a lane (dispatcher thread only).
void launch(flic_server_ctx* s, Lane& ln, std::vector<Request>& take, std::vector<int>& slots) {
    Flight& f = ln.f;
    f.reqs.swap(take);
    f.slots.swap(slots);
    f.done.store(0);
    f.t_done.store(0.0);
    f.status = FLIC_OK;
    f.cv = &s->cv;
    f.t_launch = now_s();
    const cudaStream_t st = ln.stream;
    const int n = (int)f.reqs.size();
    std::vector<flic_handle> hs(n);
    std::vector<const float*> rs(n);
    std::vector<int32_t*> ls(n);
    flic_status status = FLIC_OK;
    auto note = [&](flic_status x) {
        if (status == FLIC_OK && x != FLIC_OK) status = x;
    };
    auto cu = [&](cudaError_t e) { note(e == cudaSuccess ? FLIC_OK : FLIC_ERR_CUDA); };
    // the clouds' projection and scatter items, in launches of up to kProjBatchItems
    std::vector<flic::ProjBatch>& pb = ln.proj;
    pb.clear();
    for (int i = 0; i < n; ++i) {
        const Request& q = f.reqs[i];
        const Slot& sl = s->slots[f.slots[i]];
        const Sensor& sn = s->sensors[q.sensor];
        const size_t npix = (size_t)sn.rows * sn.cols;
        if (q.kind == 0) {
            cu(cudaMemcpyAsync(sl.d_range, q.in, npix * 4, cudaMemcpyHostToDevice, st));
        } else {
            if (q.n > 0)
                cu(cudaMemcpyAsync(sl.d_xyz, q.in, (size_t)q.n * 12, cudaMemcpyHostToDevice, st));
            if (pb.empty() || pb.back().nitems == flic::kProjBatchItems) {
                pb.emplace_back();
                pb.back().nitems = pb.back().max_n = pb.back().max_px = 0;
            }
            flic::ProjBatch& b = pb.back();
            flic::ProjItem& it = b.item[b.nitems];
            const flic_status ps = flic::proj_item(sl.h, sl.d_xyz, q.n, sl.d_range, sl.d_pix,
                                                   sl.d_labels, sl.d_plab, &it);
            note(ps);
            if (ps == FLIC_OK) {
                ++b.nitems;
                b.max_n = std::max(b.max_n, it.n);
                b.max_px = std::max(b.max_px, sn.rows * sn.cols);
            }
        }
        hs[i] = sl.h;
        rs[i] = sl.d_range;
        ls[i] = sl.d_labels;
    }
    for (const flic::ProjBatch& b : pb) cu(flic::launch_project_batch(b, st));
    size_t px = 0;
    for (int i = 0; i < n; ++i) {
        const Sensor& sn = s->sensors[f.reqs[i].sensor];
        px += (size_t)sn.rows * sn.cols;
    }
    // small strips only for a small batch on an otherwise idle GPU: under load the lanes'
    // batches share the SMs, and batch-sized strips do the work with less overhead
    bool alone = true;
    for (const Lane& o : s->lanes)
        if (&o != &ln && o.busy) alone = false;
    note(flic_label_batch(alone && px < s->small_px ? ln.batch_small : ln.batch, hs.data(),
                          rs.data(), ls.data(), n, st));
    for (const flic::ProjBatch& b : pb) cu(flic::launch_scatter_batch(b, st));
    for (int i = 0; i < n; ++i) {
        const Request& q = f.reqs[i];
        const Slot& sl = s->slots[f.slots[i]];
        const Sensor& sn = s->sensors[q.sensor];
        if (q.kind == 0) {
            cu(cudaMemcpyAsync(q.out, sl.d_labels, (size_t)sn.rows * sn.cols * 4,
                               cudaMemcpyDeviceToHost, st));
        } else if (q.n > 0) {
            cu(cudaMemcpyAsync(q.out, sl.d_plab, (size_t)q.n * 4, cudaMemcpyDeviceToHost, st));
        }
    }
    f.status = status;
    if (cudaLaunchHostFunc(st, on_batch_done, &f) != cudaSuccess) {
        cudaGetLastError();
        f.status = FLIC_ERR_CUDA;
        f.t_done.store(now_s());
        f.done.store(1);
    }
    ln.busy = true;
}

void dispatch_loop(flic_server_ctx* s) {
    cudaSetDevice(s->device);
    std::vector<Request> take;
    std::vector<int> slots;
    while (true) {
        bool did = false;
        // retire finished batches: completion records, slots back to their sensors
        for (Lane& ln : s->lanes) {
            if (!ln.busy || !ln.f.done.load()) continue;
            std::lock_guard<std::mutex> g(s->mu);
            const int n = (int)ln.f.reqs.size();
            for (int i = 0; i < n; ++i) {
                const Request& q = ln.f.reqs[i];
                flic_completion c{};
                c.tag = q.tag;
                c.sensor = q.sensor;
                c.kind = q.kind;
                c.n = q.n;
                c.status = ln.f.status;
                c.batch_size = n;
                c.t_submit = q.t_submit;
                c.t_launch = ln.f.t_launch;
                c.t_done = ln.f.t_done.load();
                s->completions.push_back(c);
                s->sensors[q.sensor].free_slots.push_back(ln.f.slots[i]);
            }
            s->completed += n;
            --s->in_flight;
            ln.busy = false;
            did = true;
            s->cv.notify_all();
        }
        // admit what has arrived into free slots and launch it on an idle lane
        Lane* idle = nullptr;
        for (Lane& ln : s->lanes)
            if (!ln.busy) {
                idle = &ln;
                break;
            }
        if (idle && !s->hold.load()) {
            take.clear();
            slots.clear();
            {
                std::lock_guard<std::mutex> g(s->mu);
                for (auto it = s->queue.begin();
                     it != s->queue.end() && (int)take.size() < s->max_batch;) {
                    std::vector<int>& fs = s->sensors[it->sensor].free_slots;
                    if (fs.empty()) {
                        ++it;
                        continue;
                    }
                    slots.push_back(fs.back());
                    fs.pop_back();
                    take.push_back(*it);
                    it = s->queue.erase(it);
                }
                if (!take.empty()) {  // in flight from the moment it leaves the queue
                    ++s->in_flight;
                    ++s->batches;
                    s->largest = std::max<int64_t>(s->largest, (int64_t)take.size());
                }
            }
            if (!take.empty()) {
                launch(s, *idle, take, slots);
                did = true;
            }
        }
        if (!did) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop.load() && (s->queue.empty() || s->hold.load()) && s->in_flight == 0) break;
            s->cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

}  // namespace

extern "C" flic_status flic_server_submit(flic_server s, int32_t sensor, int32_t kind,
                                          const void* host_in, int64_t n, int32_t* host_out,
                                          uint64_t tag) {
    if (!s || sensor < 0 || sensor >= (int)s->sensors.size() || (kind != 0 && kind != 1))
        return srv_fail(FLIC_ERR_INVALID, "flic_server_submit: bad sensor or kind");
    const Sensor& sn = s->sensors[sensor];
    if (kind == 1 && (n < 0 || n > sn.max_points))
        return srv_fail(FLIC_ERR_INVALID, "flic_server_submit: point count beyond max_points");
    if (kind == 0) n = (int64_t)sn.rows * sn.cols;
    if ((n > 0 || kind == 0) && (!host_in || !host_out))
        return srv_fail(FLIC_ERR_INVALID, "flic_server_submit: NULL buffer");
    Request q;
    q.sensor = sensor;
    q.kind = kind;
    q.in = host_in;
    q.n = n;
    q.out = host_out;
    q.tag = tag;
    q.t_submit = now_s();
    std::lock_guard<std::mutex> g(s->mu);
    if ((int)s->queue.size() >= s->max_queue) {
        ++s->rejected;
        return srv_fail(FLIC_ERR_BUSY, "flic_server_submit: admission queue full");
    }
    s->queue.push_back(q);
    ++s->submitted;
    s->cv.notify_all();
    return FLIC_OK;
}

extern "C" flic_status flic_server_hold(flic_server s, int32_t hold) {
    if (!s) return srv_fail(FLIC_ERR_INVALID, "flic_server_hold: NULL server");
    s->hold.store(hold != 0);
    s->cv.notify_all();
    return FLIC_OK;
}

extern "C" int32_t flic_server_poll(flic_server s, flic_completion* out, int32_t max) {
    if (!s || !out || max <= 0) return 0;
    std::lock_guard<std::mutex> g(s->mu);
    const int k = std::min<int>(max, (int)s->completions.size());
    std::copy(s->completions.begin(), s->completions.begin() + k, out);
    s->completions.erase(s->completions.begin(), s->completions.begin() + k);
    return k;
}

extern "C" flic_status flic_server_drain(flic_server s, double timeout_s) {
    if (!s) return srv_fail(FLIC_ERR_INVALID, "flic_server_drain: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
        return s->queue.empty() && s->in_flight == 0;
    });
    return ok ? FLIC_OK : srv_fail(FLIC_ERR_TIMEOUT, "flic_server_drain: frames still pending");
}

extern "C" flic_status flic_server_stats(flic_server s, int64_t* out) {
    if (!s || !out) return srv_fail(FLIC_ERR_INVALID, "flic_server_stats: NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    out[0] = s->submitted;
    out[1] = s->rejected;
    out[2] = s->completed;
    out[3] = s->batches;
    out[4] = s->largest;
    out[5] = (int64_t)s->slots.size();
    out[6] = s->slot_bytes;
    out[7] = s->in_flight;
    return FLIC_OK;
}

extern "C" flic_status flic_server_destroy(flic_server s) {
    if (!s) return FLIC_OK;
    s->hold.store(false);
    flic_status st = flic_server_drain(s, 30.0);
    s->stop.store(true);
    s->cv.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    cudaDeviceSynchronize();
    free_server(s);
    return st;
}
