// Continuous-batching request loop for map-making solves (bm_serve_*).
//
// max_slots worker threads, each owning a context with its own non-blocking
// CUDA stream: a worker takes the request at the head of the FIFO queue as
// soon as the head's estimated device memory fits in the remaining budget,
// runs the whole solve (ingest, noise model, preconditioner, PCG) on its
// stream, releases the memory and takes the next one.  Several requests are
// therefore resident and running on the device at once, and a request that
// arrives while others run is admitted as soon as a slot and memory free up.
// Each request's solve is exactly the single-request computation on its own
// context, so its map is bitwise the same alone and in the mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "bm_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

enum class JobState { Queued, Running, Done };

struct Job {
    uint64_t ticket = 0;
    bm_request req{};
    std::vector<int64_t> det_off;
    std::vector<double> inv_var;
    std::vector<double> coeffs;
    int64_t bytes = 0;
    JobState state = JobState::Queued;
    bm_result res{};
    Clock::time_point t_submit, t_start, t_done;
};

// Device memory a request needs while it runs (pointing, ingest scratch,
// preconditioner, solver work vectors), with a margin.
int64_t estimate_bytes(const bm_request& r) {
    const int64_t ns = r.nsamples, np = r.npix, nc = (int64_t)r.solver;
    const bool trig = r.cos2psi != nullptr;
    int64_t per_sample = 4 + 4 + (trig ? 16 : 32);  // pix, perm, trig (time + sorted; hi [+ lo])
    per_sample += 16;                               // radix-sort scratch during ingest
    // white: the weighted stream; Toeplitz: the filter's time-ordered y and
    // z (FP32 and FP64) and the chunk-major order of the inner transpose
    // (each sample's position and trig pair)
    per_sample += (r.noise == BM_NOISE_WHITE) ? 8 : 24 + 12;
    const int64_t per_pixel = 12 + 2 * 8 * nc * nc + 9 + 8 + 16 + 12 * 8 * nc;
    int64_t tmp = 0;  // the chunk-major order's build tables (at most 4 GiB, else not built)
    if (r.noise == BM_NOISE_TOEPLITZ) tmp = std::min<int64_t>(((ns >> 24) + 1) * 16 * np + 8 * np, int64_t(1) << 32);
    return ns * per_sample + np * per_pixel + tmp + (int64_t(64) << 20);
}

}  // namespace

struct bm_server {
    int device = 0;
    int64_t budget = 0;
    int max_slots = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Job> jobs;
    std::vector<std::thread> workers;
    bool stopping = false;
    uint64_t next_ticket = 1;
    int64_t reserved = 0, peak_reserved = 0;
    int64_t submitted = 0, completed = 0, rejected = 0, cancelled = 0, running = 0;
    double samples_done = 0.0;
    std::vector<double> latencies;
    Clock::time_point t_create;
};

namespace {

bm_status run_request(bm_context* ctx, Job& job) {
    const bm_request& r = job.req;
    bm_pointing* p = nullptr;
    bm_inv_noise* n = nullptr;
    bm_precond* pc = nullptr;
    bm_status st;
    if (r.cos2psi)
        st = bm_pointing_create_trig(ctx, r.npix, r.nsamples, r.pix, r.cos2psi, r.sin2psi, r.solver, &p);
    else
        st = bm_pointing_create(ctx, r.npix, r.nsamples, r.pix, r.psi, r.psi_dtype, r.solver, &p);
    if (st == BM_OK) {
        if (r.noise == BM_NOISE_WHITE)
            st = bm_inv_noise_create_diag(ctx, r.ndet, job.det_off.data(), job.inv_var.data(), &n);
        else
            st = bm_inv_noise_create_toeplitz(ctx, r.ndet, job.det_off.data(), r.chunk_len, r.nlags,
                                              job.coeffs.data(), job.inv_var.data(), &n);
    }
    if (st == BM_OK) st = bm_blockdiag_precond_create(p, n, r.min_hits, r.max_cond, &pc);
    bm_solve_info info{};
    if (st == BM_OK) {
        st = bm_pcg_solve(p, n, pc, r.tod, r.tod_dtype, 1, r.map_out, r.tol, r.maxiter, r.precision, &info);
        job.res.iterations = info.iterations;
        job.res.outer_iterations = info.outer_iterations;
        job.res.rel_residual = info.rel_residual;
    }
    bm_precond_destroy(pc);
    bm_inv_noise_destroy(n);
    bm_pointing_destroy(p);
    // Give the request's scratch back (the budget accounts per request).
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->ws.clear();
    return st;
}

void worker_main(bm_server* s, int slot) {
    cudaSetDevice(s->device);
    cudaStream_t stream = nullptr;
    bm_context* ctx = nullptr;
    bool ok = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess &&
              bm_context_create(s->device, stream, &ctx) == BM_OK;
    // A worker's scratch comes from the device's default pool: released per
    // request (the budget accounts per request) into memory that the other
    // workers and the next request reuse without mapping it again.
    if (ok && ctx->ws_pool) {
        cudaMemPoolDestroy(ctx->ws_pool);
        ctx->ws_pool = nullptr;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        s->cv_work.wait(lk, [&] {
            return s->stopping ||
                   (!s->queue.empty() && s->reserved + s->jobs[s->queue.front()].bytes <= s->budget);
        });
        if (s->stopping) break;
        const uint64_t t = s->queue.front();
        s->queue.pop_front();
        Job& job = s->jobs[t];
        job.state = JobState::Running;
        job.t_start = Clock::now();
        job.res.slot = slot;
        s->reserved += job.bytes;
        s->peak_reserved = std::max(s->peak_reserved, s->reserved);
        s->running += 1;
        lk.unlock();
        const bm_status st = ok ? run_request(ctx, job) : BM_ERR_CUDA;
        char msg[sizeof(job.res.message)] = "";
        if (st != BM_OK) std::snprintf(msg, sizeof(msg), "%s", ok ? bm_last_error() : "worker context failed");
        lk.lock();
        job.t_done = Clock::now();
        job.res.status = st;
        std::memcpy(job.res.message, msg, sizeof(msg));
        job.res.queue_ms = ms_between(job.t_submit, job.t_start);
        job.res.run_ms = ms_between(job.t_start, job.t_done);
        job.res.latency_ms = ms_between(job.t_submit, job.t_done);
        job.res.device_bytes = job.bytes;
        job.state = JobState::Done;
        s->reserved -= job.bytes;
        s->running -= 1;
        s->completed += 1;
        s->samples_done += (double)job.req.nsamples;
        s->latencies.push_back(job.res.latency_ms);
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    lk.unlock();
    if (ctx) bm_context_destroy(ctx);
    if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

bm_status bm_serve_create(bm_context* ctx, size_t hbm_budget_bytes, int32_t max_slots, bm_server** out) {
    bm::clear_error();
    if (!ctx || !out) { bm::set_error("ctx/out is NULL"); return BM_ERR_INVALID; }
    *out = nullptr;
    if (max_slots < 1 || max_slots > 64) { bm::set_error("max_slots %d out of [1, 64]", max_slots); return BM_ERR_INVALID; }
    if (hbm_budget_bytes == 0) { bm::set_error("zero memory budget"); return BM_ERR_INVALID; }
    bm_server* s = new (std::nothrow) bm_server();
    if (!s) { bm::set_error("host allocation failed"); return BM_ERR_OOM; }
    s->device = ctx->device;
    s->budget = (int64_t)std::min<size_t>(hbm_budget_bytes, (size_t)INT64_MAX);
    s->max_slots = max_slots;
    s->t_create = Clock::now();
    try {
        for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker_main, s, i);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stopping = true;
        }
        s->cv_work.notify_all();
        for (auto& w : s->workers) w.join();
        delete s;
        bm::set_error("could not start the worker threads");
        return BM_ERR_CUDA;
    }
    *out = s;
    return BM_OK;
}

bm_status bm_serve_submit(bm_server* s, const bm_request* req, uint64_t* ticket) {
    bm::clear_error();
    if (!s || !req || !ticket) { bm::set_error("NULL argument"); return BM_ERR_INVALID; }
    const bm_request& r = *req;
    if (r.npix < 1 || r.nsamples < 1 || !r.pix || !r.tod || !r.map_out || r.ndet < 1 || !r.det_offsets ||
        !r.inv_var || (!r.cos2psi && !r.psi) || (r.cos2psi && !r.sin2psi) ||
        (r.noise == BM_NOISE_TOEPLITZ && (!r.coeffs || r.nlags < 1 || r.chunk_len < 1)) ||
        (r.solver != BM_SOLVER_I && r.solver != BM_SOLVER_QU && r.solver != BM_SOLVER_IQU) ||
        r.det_offsets[r.ndet] != r.nsamples) {
        bm::set_error("malformed request");
        return BM_ERR_INVALID;
    }
    Job job;
    job.req = r;
    job.det_off.assign(r.det_offsets, r.det_offsets + r.ndet + 1);
    job.inv_var.assign(r.inv_var, r.inv_var + r.ndet);
    if (r.noise == BM_NOISE_TOEPLITZ) job.coeffs.assign(r.coeffs, r.coeffs + (size_t)r.ndet * r.nlags);
    job.req.det_offsets = nullptr;
    job.req.inv_var = nullptr;
    job.req.coeffs = nullptr;
    job.bytes = estimate_bytes(r);
    job.t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    s->submitted += 1;
    if (s->stopping) { bm::set_error("server is shutting down"); return BM_ERR_BUSY; }
    if (job.bytes > s->budget) {
        s->rejected += 1;
        bm::set_error("request needs about %lld bytes, more than the whole budget of %lld",
                      (long long)job.bytes, (long long)s->budget);
        return BM_ERR_BUSY;
    }
    const uint64_t t = s->next_ticket++;
    job.ticket = t;
    s->jobs.emplace(t, std::move(job));
    s->queue.push_back(t);
    *ticket = t;
    s->cv_work.notify_all();
    return BM_OK;
}

bm_status bm_serve_poll(bm_server* s, uint64_t ticket, int32_t timeout_ms, bm_result* out) {
    bm::clear_error();
    if (!s) { bm::set_error("NULL server"); return BM_ERR_INVALID; }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) { bm::set_error("unknown ticket %llu", (unsigned long long)ticket); return BM_ERR_NOT_FOUND; }
    const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    while (it->second.state != JobState::Done) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            it = s->jobs.find(ticket);
            if (it == s->jobs.end()) return BM_ERR_NOT_FOUND;
            if (it->second.state != JobState::Done) return BM_ERR_TIMEOUT;
            break;
        }
        it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return BM_ERR_NOT_FOUND;
    }
    if (out) *out = it->second.res;
    s->jobs.erase(it);
    return BM_OK;
}

bm_status bm_serve_cancel(bm_server* s, uint64_t ticket) {
    bm::clear_error();
    if (!s) { bm::set_error("NULL server"); return BM_ERR_INVALID; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return BM_ERR_NOT_FOUND;
    if (it->second.state != JobState::Queued) return BM_ERR_BUSY;
    s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), ticket), s->queue.end());
    Job& j = it->second;
    j.state = JobState::Done;
    j.res.status = BM_ERR_NOT_FOUND;
    j.t_done = Clock::now();
    j.res.latency_ms = ms_between(j.t_submit, j.t_done);
    s->cancelled += 1;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    return BM_OK;
}

bm_status bm_serve_get_stats(bm_server* s, bm_serve_stats* out) {
    bm::clear_error();
    if (!s || !out) { bm::set_error("NULL argument"); return BM_ERR_INVALID; }
    std::lock_guard<std::mutex> lk(s->mu);
    bm_serve_stats st{};
    st.submitted = s->submitted;
    st.completed = s->completed;
    st.rejected = s->rejected;
    st.cancelled = s->cancelled;
    st.running = s->running;
    st.queued = (int64_t)s->queue.size();
    std::vector<double> l = s->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            const size_t i = (size_t)std::min<double>((double)l.size() - 1, std::ceil(q * l.size()) - 1);
            return l[i];
        };
        st.p50_ms = pct(0.50);
        st.p99_ms = pct(0.99);
        double sum = 0.0;
        for (double v : l) sum += v;
        st.mean_ms = sum / (double)l.size();
    }
    const double wall_s = ms_between(s->t_create, Clock::now()) / 1e3;
    st.samples_per_s = wall_s > 0 ? s->samples_done / wall_s : 0.0;
    st.budget_bytes = s->budget;
    st.reserved_bytes = s->reserved;
    st.peak_reserved_bytes = s->peak_reserved;
    *out = st;
    return BM_OK;
}

void bm_serve_destroy(bm_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        for (uint64_t t : s->queue) {
            Job& j = s->jobs[t];
            j.state = JobState::Done;
            j.res.status = BM_ERR_NOT_FOUND;
            s->cancelled += 1;
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (auto& w : s->workers) w.join();
    // the workers' memory went back to the device's default pool, which
    // keeps it cached: hand it back to the device
    cudaMemPool_t pool = nullptr;
    if (cudaSetDevice(s->device) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
        cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess)
        cudaMemPoolTrimTo(pool, 0);
    delete s;
}

}  // extern "C"
