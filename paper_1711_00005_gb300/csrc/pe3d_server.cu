// pe3d_server.cu -- the request loop: continuous batching of independent
// marches (the paper's multi-frequency farm, Fig. 2's frequency loop, Sec.
// 3.2.3) on one GPU.
//
// Two host threads:
//   * the admission thread takes queued requests in arrival order while the
//     device-memory budget and the active-march limit allow, and sets each up
//     on a stream of its own (plan, medium upload with FP64 set-up, per-step
//     azimuth set-up, prologue, status check), then hands it to the
//     scheduler's ready list;
//   * the scheduler thread owns the batch stream.  Each turn it moves ready
//     requests into the batch, advances every admitted march by up to `chunk`
//     range steps in shared batched launches (one per precision, at most 64
//     marches each), and retires finished marches (copies their snapshots to
//     host memory and releases their device memory, so waiting requests can
//     be admitted).
// A request's set-up thus never stalls the marches already running: the
// scheduler waits on nothing but its own launches.  Requests that arrive
// while others run join at the turn after their set-up ends.  The per-system
// arithmetic does not depend on who else is in the batch, so a request's
// result is the same alone and in the mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pe3d_internal.h"
#include "pe3d_kernels.cuh"

namespace pe3d_host {
int serve_begin_f32(pe3d_plan_s* p, const void* u0_dev, double r0, int steps, int stride, void* snap_dev,
                    pe3d::MarchArgs<float2>* desc);
int serve_tick_f32(pe3d_plan_s* owner, pe3d::MarchArgs<float2>* descs, int n, int nsteps);
int serve_begin_f64(pe3d_plan_s* p, const void* u0_dev, double r0, int steps, int stride, void* snap_dev,
                    pe3d::MarchArgs<double2>* desc);
int serve_tick_f64(pe3d_plan_s* owner, pe3d::MarchArgs<double2>* descs, int n, int nsteps);
}  // namespace pe3d_host

using namespace pe3d_host;

namespace {

struct Request {
    uint64_t id = 0;
    pe3d_request r{};
    std::vector<unsigned char> n2, u0;    // owned copies of the inputs
    std::vector<double> slice_r;
    std::vector<unsigned char> out;       // host snapshots once done
    int state = PE3D_REQ_PENDING;
    double t_submit = 0, t_start = 0, t_done = 0;
    size_t est_bytes = 0;
    pe3d_plan_t plan = nullptr;
    cudaStream_t stream = nullptr;        // the request's set-up stream
    void* u0_dev = nullptr;
    void* snap_dev = nullptr;
    size_t snap_bytes = 0;
    int j = 0;                            // next range step
    pe3d::MarchArgs<float2> d32;
    pe3d::MarchArgs<double2> d64;
    std::string error;
};

size_t elem_of(int precision) { return precision == PE3D_FP32 ? 8 : 16; }

}  // namespace

struct pe3d_server_s {
    size_t budget = 0;
    int max_active = 64;
    int chunk = 64;
    int device = 0;
    cudaStream_t stream = nullptr;
    pe3d_plan_t owner = nullptr;          // barrier, status and descriptor buffer of the batched launches
    std::thread th;                       // scheduler
    std::thread admit_th;                 // admission
    std::mutex mu;
    std::condition_variable cv;           // wakes the admission thread (new request, freed memory, stop)
    std::condition_variable cv_ready;     // wakes the scheduler (a request is set up, stop)
    bool stop = false;
    std::deque<Request*> pending;
    std::deque<Request*> ready;           // set up, joining the batch at the next turn
    std::vector<Request*> active;
    int setting_up = 0;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
    uint64_t next_id = 1;
    size_t used = 0;
    std::chrono::steady_clock::time_point t0;
    int64_t n_submitted = 0, n_admitted = 0, n_finished = 0, n_failed = 0, n_ticks = 0, point_steps = 0;
    int64_t setup_launches = 0;           // kernels the admission thread launched (set-up of each request)
    int64_t tick_launches = 0;            // kernels of the batched turns (the owner plan's count)
    int64_t tick_us = 0;                  // scheduler time in turns (launch, wait, retire)
    int64_t kernel_us = 0;                // GPU time of the turns' launches (events on the server stream)
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    void loop();
    void admit_loop();
    bool start(Request* q);
    void finish(Request* q, bool ok, const std::string& why);
    bool tick();
};

// Device bytes a request will hold while it runs (plan buffers, medium,
// coefficients, per-step tables, snapshots); the layout is the library's.
static int estimate_bytes(const pe3d_request& r, size_t* out) {
    pe3d_plan_s tmp;
    tmp.Nz = r.Nz; tmp.Nt = r.Ntheta; tmp.precision = r.precision; tmp.boundary = r.boundary;
    int rc = r.precision == PE3D_FP32 ? layout_choose_f32(&tmp) : layout_choose_f64(&tmp);
    if (rc) return rc;
    const size_t es = elem_of(r.precision);
    const size_t field = (size_t)r.Ntheta * tmp.ldz * es;
    const size_t pts = (size_t)r.Ntheta * r.Nz;
    size_t b = 2 * field + (size_t)r.K * pts * 16 + (size_t)r.K * field + pts * es;
    const size_t steps = (size_t)std::max(r.steps, 1);
    b += steps * tmp.NtP * es * (r.boundary == PE3D_PERIODIC ? 2 : 1) + steps * (sizeof(pe3d::StepConst) + 4);
    if (r.boundary == PE3D_PERIODIC) b += 2 * steps * tmp.NtP * 16;
    b += (size_t)(r.steps / r.out_stride) * pts * es;
    if (r.rc_every > 0) b += 3 * field;   // u^j, the uncorrected u^{j+1} and the correction
    *out = b + 4096;
    return PE3D_OK;
}

// Set a request up on its own stream (admission thread); true when it can join
// the batch.  Ends with a synchronisation of that stream only.
bool pe3d_server_s::start(Request* q) {
    const pe3d_request& r = q->r;
    cudaError_t se = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking);
    if (se != cudaSuccess) {
        q->stream = nullptr;
        finish(q, false, std::string("request stream: ") + cudaGetErrorString(se));
        return false;
    }
    cudaStream_t stream = q->stream;
    int rc = pe3d_plan(r.Nz, r.Ntheta, r.dz, r.dtheta, r.dr, r.k0, r.boundary, r.precision, stream, &q->plan);
    if (!rc && r.rc_every > 0) rc = pe3d_set_option(q->plan, PE3D_OPT_RC_EVERY, r.rc_every);
    if (!rc) rc = pe3d_set_medium(q->plan, q->n2.data(), q->slice_r.data(), r.K, 0);
    const size_t es = elem_of(r.precision);
    const size_t fbytes = (size_t)r.Ntheta * r.Nz * es;
    const int n_out = r.steps / r.out_stride;
    if (!rc) rc = dev_alloc(q->plan, &q->u0_dev, fbytes);
    if (!rc && n_out > 0) {
        q->snap_bytes = (size_t)n_out * fbytes;
        rc = dev_alloc(q->plan, &q->snap_dev, q->snap_bytes);
    }
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(q->u0_dev, q->u0.data(), fbytes, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "u0 upload");
    }
    if (!rc) {
        rc = r.precision == PE3D_FP32
                 ? serve_begin_f32(q->plan, q->u0_dev, r.r0, r.steps, r.out_stride, q->snap_dev, &q->d32)
                 : serve_begin_f64(q->plan, q->u0_dev, r.r0, r.steps, r.out_stride, q->snap_dev, &q->d64);
    }
    if (!rc) {
        int st = 0;
        cudaError_t e = cudaMemcpyAsync(&st, q->plan->status, sizeof(int), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "request set-up");
        else if (st) rc = fail(st, "singular system in the request's azimuth set-up");
    }
    if (q->plan) {
        std::lock_guard<std::mutex> lk(mu);
        setup_launches += q->plan->total_launches;
    }
    if (rc) {
        finish(q, false, pe3d_last_error());
        return false;
    }
    std::vector<unsigned char>().swap(q->n2);   // the medium now lives on the device
    q->j = 0;
    return true;
}

void pe3d_server_s::finish(Request* q, bool ok, const std::string& why) {
    if (ok && q->snap_bytes) {
        q->out.resize(q->snap_bytes);
        cudaError_t e = cudaMemcpy(q->out.data(), q->snap_dev, q->snap_bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { ok = false; q->error = cudaGetErrorString(e); }
    }
    if (q->plan) {
        dev_free(q->plan, &q->u0_dev, 0);
        dev_free(q->plan, &q->snap_dev, 0);
        pe3d_destroy(q->plan);
        q->plan = nullptr;
    }
    if (q->stream) {
        cudaStreamDestroy(q->stream);
        q->stream = nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    used -= std::min(used, q->est_bytes);
    q->t_done = now();
    q->state = ok ? PE3D_REQ_DONE : PE3D_REQ_FAILED;
    if (!ok && q->error.empty()) q->error = why;
    if (ok) {
        ++n_finished;
        point_steps += (int64_t)q->r.Nz * q->r.Ntheta * q->r.steps;
    } else {
        ++n_failed;
    }
}

// Advance every active march by up to `chunk` steps; retire finished ones.
bool pe3d_server_s::tick() {
    std::vector<Request*> act;
    {
        std::lock_guard<std::mutex> lk(mu);
        act = active;
    }
    if (act.empty()) return false;
    const auto tw0 = std::chrono::steady_clock::now();
    bool ok = true;
    std::string why;
    cudaEventRecord(ev_a, stream);
    for (int prec : {PE3D_FP32, PE3D_FP64}) {
        std::vector<Request*> grp;
        for (Request* q : act)
            if (q->r.precision == prec && q->j < q->r.steps) grp.push_back(q);
        for (size_t b = 0; b < grp.size() && ok; b += pe3d::BATCH_MAX) {
            const size_t e = std::min(grp.size(), b + pe3d::BATCH_MAX);
            int nsteps = 0, rc = 0;
            if (prec == PE3D_FP32) {
                std::vector<pe3d::MarchArgs<float2>> d;
                for (size_t i = b; i < e; ++i) {
                    Request* q = grp[i];
                    q->d32.j0 = q->j;
                    q->d32.j1 = std::min(q->j + chunk, q->r.steps);
                    nsteps = std::max(nsteps, q->d32.j1 - q->d32.j0);
                    d.push_back(q->d32);
                }
                rc = serve_tick_f32(owner, d.data(), (int)d.size(), nsteps);
            } else {
                std::vector<pe3d::MarchArgs<double2>> d;
                for (size_t i = b; i < e; ++i) {
                    Request* q = grp[i];
                    q->d64.j0 = q->j;
                    q->d64.j1 = std::min(q->j + chunk, q->r.steps);
                    nsteps = std::max(nsteps, q->d64.j1 - q->d64.j0);
                    d.push_back(q->d64);
                }
                rc = serve_tick_f64(owner, d.data(), (int)d.size(), nsteps);
            }
            if (rc) { ok = false; why = pe3d_last_error(); }
            // the descriptor buffer is reused by the next launch: wait here
            cudaError_t ce = cudaStreamSynchronize(stream);
            if (ce != cudaSuccess) { ok = false; why = cudaGetErrorString(ce); }
        }
    }
    cudaEventRecord(ev_b, stream);
    int st = 0;
    if (ok) {
        cudaError_t ce = cudaMemcpy(&st, owner->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess || st != 0) { ok = false; why = "device status " + std::to_string(st); }
    }
    float kms = 0.f;
    if (cudaEventSynchronize(ev_b) != cudaSuccess || cudaEventElapsedTime(&kms, ev_a, ev_b) != cudaSuccess) {
        cudaGetLastError();
        kms = 0.f;
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        ++n_ticks;
        tick_launches = owner->total_launches;
        kernel_us += (int64_t)(kms * 1e3f);
    }
    std::vector<Request*> done;
    for (Request* q : act) {
        if (!ok) { done.push_back(q); continue; }
        q->j = std::min(q->j + chunk, q->r.steps);
        if (q->j >= q->r.steps) done.push_back(q);
    }
    for (Request* q : done) {
        {
            std::lock_guard<std::mutex> lk(mu);
            active.erase(std::remove(active.begin(), active.end(), q), active.end());
        }
        finish(q, ok, why);
    }
    if (!ok) {   // clear the status word for the next batch
        cudaMemset(owner->status, 0, sizeof(int));
    }
    if (!done.empty()) cv.notify_all();   // memory freed: the admission thread may take the next request
    {
        std::lock_guard<std::mutex> lk(mu);
        tick_us += std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - tw0)
                       .count();
    }
    return true;
}

// Admission thread: in arrival order, while the budget and the active-march
// limit allow (a request larger than the budget still runs when nothing else
// holds memory), set the next request up and put it on the ready list.
void pe3d_server_s::admit_loop() {
    cudaSetDevice(device);
    for (;;) {
        Request* q = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] {
                if (stop) return true;
                if (pending.empty()) return false;
                const int in_flight = (int)active.size() + (int)ready.size() + setting_up;
                const bool empty = in_flight == 0;
                return in_flight < max_active && (used + pending.front()->est_bytes <= budget || empty);
            });
            if (stop) return;
            q = pending.front();
            pending.pop_front();
            used += q->est_bytes;
            q->state = PE3D_REQ_RUNNING;
            q->t_start = now();
            ++n_admitted;
            ++setting_up;
        }
        const bool ok = start(q);
        {
            std::lock_guard<std::mutex> lk(mu);
            --setting_up;
            if (ok) ready.push_back(q);
        }
        cv_ready.notify_all();
        cv.notify_all();   // a failed set-up released its memory
    }
}

// Scheduler thread: join the ready requests, one turn of the batched march,
// retire; wait when there is nothing to march.
void pe3d_server_s::loop() {
    cudaSetDevice(device);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(mu);
            if (stop) return;
            while (!ready.empty()) {
                active.push_back(ready.front());
                ready.pop_front();
            }
        }
        if (!tick()) {
            std::unique_lock<std::mutex> lk(mu);
            cv_ready.wait_for(lk, std::chrono::milliseconds(5), [&] { return stop || !ready.empty(); });
            if (stop) return;
        }
    }
}

extern "C" {

int pe3d_server_create(size_t mem_budget, int max_active, int chunk, pe3d_server_t* out) {
    set_error("");
    if (!out) return fail(PE3D_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (mem_budget == 0 || max_active < 1 || chunk < 1) return fail(PE3D_ERR_ARG, "budget, max_active, chunk must be > 0");
    std::unique_ptr<pe3d_server_s> s(new (std::nothrow) pe3d_server_s());
    if (!s) return fail(PE3D_ERR_OOM, "host allocation failed");
    s->budget = mem_budget;
    s->max_active = max_active;
    s->chunk = chunk;
    s->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev_a);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev_b);
    if (e != cudaSuccess) {
        if (s->ev_a) cudaEventDestroy(s->ev_a);
        if (s->stream) cudaStreamDestroy(s->stream);
        return cuda_fail(e, "server stream");
    }
    int rc = pe3d_plan(1, 1, 1.0, 1.0, 1.0, 1.0, PE3D_WALLED, PE3D_FP32, s->stream, &s->owner);
    if (rc) {
        cudaEventDestroy(s->ev_a);
        cudaEventDestroy(s->ev_b);
        cudaStreamDestroy(s->stream);
        return rc;
    }
    pe3d_server_s* raw = s.release();
    raw->th = std::thread([raw] { raw->loop(); });
    raw->admit_th = std::thread([raw] { raw->admit_loop(); });
    *out = raw;
    return PE3D_OK;
}

int pe3d_submit(pe3d_server_t s, const pe3d_request* r, uint64_t* id) {
    set_error("");
    if (!s || !r || !id) return fail(PE3D_ERR_ARG, "NULL argument");
    if (r->Nz < 1 || r->Ntheta < 1 || r->K < 1 || r->steps < 0 || r->out_stride < 1 || !(r->r0 > 0) ||
        !r->n2 || !r->slice_r || !r->u0 || (r->precision != PE3D_FP32 && r->precision != PE3D_FP64) ||
        (r->boundary != PE3D_WALLED && r->boundary != PE3D_PERIODIC) ||
        (r->boundary == PE3D_PERIODIC && r->Ntheta < 3) || !(r->dz > 0) || !(r->dtheta > 0) || !(r->k0 > 0) ||
        !(r->dr != 0))
        return fail(PE3D_ERR_ARG, "invalid request");
    if (r->rc_every < 0 || (r->rc_every > 0 && r->precision != PE3D_FP32))
        return fail(PE3D_ERR_ARG, "rc_every must be >= 0, and the FP64 residual correction is for FP32 requests");
    for (int k = 1; k < r->K; ++k)
        if (!(r->slice_r[k] > r->slice_r[k - 1])) return fail(PE3D_ERR_ARG, "slice ranges must ascend");
    size_t est = 0;
    int rc = estimate_bytes(*r, &est);
    if (rc) return rc;
    if (est > s->budget) return fail(PE3D_ERR_ARG, "request needs " + std::to_string(est) +
                                                       " device bytes, more than the server's budget");
    std::unique_ptr<Request> q(new (std::nothrow) Request());
    if (!q) return fail(PE3D_ERR_OOM, "host allocation failed");
    const size_t pts = (size_t)r->Ntheta * r->Nz;
    try {
        q->n2.assign((const unsigned char*)r->n2, (const unsigned char*)r->n2 + (size_t)r->K * pts * 16);
        q->u0.assign((const unsigned char*)r->u0, (const unsigned char*)r->u0 + pts * elem_of(r->precision));
        q->slice_r.assign(r->slice_r, r->slice_r + r->K);
    } catch (...) {
        return fail(PE3D_ERR_OOM, "host allocation failed");
    }
    q->r = *r;
    q->r.n2 = nullptr; q->r.u0 = nullptr; q->r.slice_r = nullptr;
    q->est_bytes = est;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        q->id = s->next_id++;
        q->t_submit = s->now();
        *id = q->id;
        s->pending.push_back(q.get());
        s->all[q->id] = std::move(q);
        ++s->n_submitted;
    }
    s->cv.notify_one();
    return PE3D_OK;
}

int pe3d_poll(pe3d_server_t s, uint64_t id, int* state, void* out, double* times) {
    set_error("");
    if (!s || !state) return fail(PE3D_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(PE3D_ERR_ARG, "unknown request id");
    Request* q = it->second.get();
    *state = q->state;
    if (times) { times[0] = q->t_submit; times[1] = q->t_start; times[2] = q->t_done; }
    if (q->state == PE3D_REQ_FAILED) {
        std::string why = q->error;
        if (out) s->all.erase(it);
        return fail(PE3D_ERR_CUDA, "request failed: " + why);
    }
    if (q->state == PE3D_REQ_DONE && out) {
        if (!q->out.empty()) std::memcpy(out, q->out.data(), q->out.size());
        s->all.erase(it);
    }
    return PE3D_OK;
}

int pe3d_server_stats(pe3d_server_t s, int64_t* stats, int n) {
    set_error("");
    if (!s || !stats || n < 0) return fail(PE3D_ERR_ARG, "bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t v[] = {s->n_submitted, s->n_admitted, s->n_finished, s->n_failed, s->n_ticks, s->point_steps,
                         (int64_t)s->used, s->setup_launches + s->tick_launches, s->tick_us, s->kernel_us};
    const int cnt = std::min<int>(n, 10);
    for (int i = 0; i < cnt; ++i) stats[i] = v[i];
    return cnt;
}

int pe3d_server_destroy(pe3d_server_t s) {
    set_error("");
    if (!s) return PE3D_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    s->cv_ready.notify_all();
    if (s->th.joinable()) s->th.join();
    if (s->admit_th.joinable()) s->admit_th.join();
    for (auto& kv : s->all) {
        Request* q = kv.second.get();
        if (q->plan) {
            dev_free(q->plan, &q->u0_dev, 0);
            dev_free(q->plan, &q->snap_dev, 0);
            pe3d_destroy(q->plan);
        }
        if (q->stream) cudaStreamDestroy(q->stream);
    }
    if (s->owner) pe3d_destroy(s->owner);
    if (s->ev_a) cudaEventDestroy(s->ev_a);
    if (s->ev_b) cudaEventDestroy(s->ev_b);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return PE3D_OK;
}

}  // extern "C"
