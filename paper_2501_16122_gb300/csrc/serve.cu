// Continuous-batching request loop for map-making solves (bm_serve_*).
//
// max_slots worker threads, each owning a context with its own non-blocking
// CUDA stream: a worker takes the first runnable request of the FIFO queue
// as soon as its estimated device memory fits in what the budget has left,
// runs it on a stream of its own, releases its scratch and takes the next
// one.  Several requests are therefore resident and running on the device at
// once, and a request that arrives while others run is admitted as soon as a
// slot and memory free up.
//
// Resident pointings.  A request with a nonzero pointing_key runs on a
// resident entry of that key: a context with its own stream that holds the
// ingested pointing, the noise model and the preconditioner.  The first
// request of a key builds the entry; it stays on the device after the
// request completes and later requests of the key skip the ingest (and the
// preconditioner, when their noise model matches).  An entry is used by one
// slot at a time: requests whose entry is in use wait (later requests may
// overtake them), and a slot that takes a white-noise mixed-precision
// request gathers every queued request of the same key and solve settings
// into one multi-RHS solve on the entry (one pass over the pointing for all
// of them).  Entries count against the budget; the least recently used idle
// entry is released when an admitted request needs the memory.
//
// A request whose allocation fails while other requests hold memory is
// queued again (at most kMaxOomRetries times) and becomes runnable once one
// of them has completed (idle resident entries are released first).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "bm_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

constexpr int kMaxOomRetries = 3;
constexpr int64_t kMargin = int64_t(64) << 20;

enum class JobState { Queued, Running, Done };

struct Job {
    uint64_t ticket = 0;
    bm_request req{};
    std::vector<int64_t> det_off;
    std::vector<double> inv_var;
    std::vector<double> coeffs;
    int64_t bytes = 0;           // reserved while it runs
    int oom_retries = 0;
    int64_t wait_completed = -1; // runnable again once completed > this (after an OOM)
    JobState state = JobState::Queued;
    bm_result res{};
    Clock::time_point t_submit, t_start, t_done;
};

// Memory model of a request (estimates with a margin; an underestimate is
// caught by the OOM re-queue).
//  resident: what the ingested pointing, the noise model and the
//            preconditioner keep (perm + sorted pixel, sorted trig pair(s),
//            the weighted stream or the chunk-major copy of the Toeplitz
//            transpose; per pixel the blocks, their inverses, mask, hits)
//  create:   scratch of building them (the radix sort's records; the
//            chunk-major order's build tables, at most 4 GiB)
//  solve(R): scratch of a solve of R right-hand sides on them (for R > 1 the
//            TOD group transposed for the batched RHS, up to 64 rows)
int64_t est_resident(const bm_request& r) {
    const int64_t ns = r.nsamples, np = r.npix, nc = (int64_t)r.solver;
    const int64_t trig = r.cos2psi != nullptr ? 16 : 32;
    const int64_t tail = r.noise == BM_NOISE_WHITE ? 8 : 12;
    return ns * (8 + trig + tail) + np * (45 + 16 * nc * nc);
}

int64_t est_create(const bm_request& r) {
    int64_t tmp = 0;
    if (r.noise == BM_NOISE_TOEPLITZ)
        tmp = std::min<int64_t>(((r.nsamples >> 24) + 1) * 16 * r.npix + 8 * r.npix, int64_t(1) << 32);
    return r.nsamples * 16 + tmp;
}

int64_t est_solve(const bm_request& r, int R) {
    const int64_t ns = r.nsamples, np = r.npix, nc = (int64_t)r.solver;
    if (R <= 1) return ns * (r.noise == BM_NOISE_WHITE ? 0 : 24) + np * 96 * nc;
    const int64_t esz = r.tod_dtype == BM_F64 ? 8 : 4;
    const int64_t items = np + ns / bm::kItemMax + 1;
    return ns * std::min(R, 64) * esz + (int64_t)R * nc * (np * (11 * 8 + 4) + items * 8);
}

// Everything the noise model and preconditioner of a request depend on.
struct NoiseSig {
    int noise = 0;
    std::vector<double> inv_var, coeffs;
    int64_t chunk_len = 0;
    int32_t nlags = 0, min_hits = 0;
    double max_cond = 0.0;
    bool operator==(const NoiseSig& o) const {
        return noise == o.noise && inv_var == o.inv_var && coeffs == o.coeffs && chunk_len == o.chunk_len &&
               nlags == o.nlags && min_hits == o.min_hits && max_cond == o.max_cond;
    }
};

NoiseSig noise_sig(const Job& j) {
    NoiseSig s;
    s.noise = (int)j.req.noise;
    s.inv_var = j.inv_var;
    s.coeffs = j.coeffs;
    if (j.req.noise == BM_NOISE_TOEPLITZ) {
        s.chunk_len = j.req.chunk_len;
        s.nlags = j.req.nlags;
    }
    s.min_hits = j.req.min_hits;
    s.max_cond = j.req.max_cond;
    return s;
}

// Requests that may share one multi-RHS solve.
bool batchable(const Job& j) {
    return j.req.pointing_key != 0 && j.req.noise == BM_NOISE_WHITE && j.req.precision == BM_PREC_MIXED;
}

bool same_batch(const Job& a, const Job& b) {
    return a.req.pointing_key == b.req.pointing_key && batchable(a) && batchable(b) &&
           a.req.npix == b.req.npix && a.req.nsamples == b.req.nsamples && a.req.solver == b.req.solver &&
           a.det_off == b.det_off && a.inv_var == b.inv_var && a.req.min_hits == b.req.min_hits &&
           a.req.max_cond == b.req.max_cond && a.req.tol == b.req.tol && a.req.maxiter == b.req.maxiter &&
           a.req.tod_dtype == b.req.tod_dtype;
}

// A resident pointing (with the noise model and preconditioner of its last
// use), on a context and stream of its own.
struct Resident {
    uint64_t key = 0;
    cudaStream_t stream = nullptr;
    bm_context* ctx = nullptr;
    bm_pointing* p = nullptr;
    bm_inv_noise* n = nullptr;
    bm_precond* pc = nullptr;
    NoiseSig sig;
    int64_t npix = 0, nsamples = 0;
    int solver = 0;
    std::vector<int64_t> det_off;
    int64_t bytes = 0;      // counted in the server's resident total once ready
    bool ready = false;     // handles built
    bool in_use = false;
    uint64_t last_use = 0;
};

void destroy_resident(Resident* e) {
    if (!e) return;
    bm_precond_destroy(e->pc);
    bm_inv_noise_destroy(e->n);
    bm_pointing_destroy(e->p);
    if (e->ctx) bm_context_destroy(e->ctx);
    if (e->stream) cudaStreamDestroy(e->stream);
    delete e;
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
    std::map<uint64_t, Resident*> resident;  // by pointing_key
    std::vector<std::thread> workers;
    bool stopping = false;
    uint64_t next_ticket = 1, tick = 0;
    int64_t reserved = 0, peak_reserved = 0, resident_total = 0;
    int64_t submitted = 0, completed = 0, rejected = 0, cancelled = 0, running = 0;
    int64_t resident_hits = 0, batches = 0, batched_requests = 0, evictions = 0, oom_requeues = 0;
    double samples_done = 0.0;
    std::vector<double> latencies;
    Clock::time_point t_create;
};

namespace {

// What a slot took from the queue: one request, or a batch of requests of
// one key, with the memory reserved for them and the idle entries released
// to make room (destroyed by the slot outside the lock).
struct Plan {
    std::vector<uint64_t> tickets;
    Resident* entry = nullptr;
    bool resident_hit = false;
    bool reject = false;   // the key names a pointing of another shape
    int64_t bytes = 0;
    std::vector<Resident*> victims;
};

int64_t evictable_bytes(const bm_server* s, const Resident* keep) {
    int64_t b = 0;
    for (const auto& kv : s->resident)
        if (kv.second != keep && kv.second->ready && !kv.second->in_use) b += kv.second->bytes;
    return b;
}

bool fits(const bm_server* s, int64_t need, const Resident* keep) {
    const int64_t used = s->reserved + s->resident_total;
    if (used + need <= s->budget) return true;
    return used - evictable_bytes(s, keep) + need <= s->budget;
}

// Release least recently used idle entries (never keep) until need fits.
void make_room(bm_server* s, int64_t need, const Resident* keep, std::vector<Resident*>& victims) {
    while (s->reserved + s->resident_total + need > s->budget) {
        Resident* lru = nullptr;
        for (const auto& kv : s->resident) {
            Resident* e = kv.second;
            if (e == keep || !e->ready || e->in_use) continue;
            if (!lru || e->last_use < lru->last_use) lru = e;
        }
        if (!lru) return;
        s->resident.erase(lru->key);
        s->resident_total -= lru->bytes;
        s->evictions += 1;
        victims.push_back(lru);
    }
}

bool shape_matches(const Resident* e, const Job& j) {
    return e->npix == j.req.npix && e->nsamples == j.req.nsamples && e->solver == (int)j.req.solver &&
           e->det_off == j.det_off;
}

// The first runnable request of the queue (with the queued requests that
// can share its solve); false when there is none, or when the first one
// does not fit in memory (it then waits: first come, first served).
// Called under the lock; changes nothing when it returns false.
bool pick(bm_server* s, Plan& plan) {
    plan = Plan{};
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        Job& j = s->jobs[*it];
        if (j.wait_completed >= 0 && s->completed <= j.wait_completed && s->running > 0) continue;
        Resident* e = nullptr;
        const uint64_t key = j.req.pointing_key;
        if (key) {
            auto f = s->resident.find(key);
            if (f != s->resident.end()) {
                e = f->second;
                if (e->in_use) continue;  // wait for the slot that uses it
                if (!shape_matches(e, j)) {
                    plan.tickets.push_back(*it);
                    plan.reject = true;
                    s->queue.erase(it);
                    return true;
                }
            }
        }
        const bool ready = e && e->ready;
        int64_t need = (ready ? 0 : est_resident(j.req) + est_create(j.req)) + est_solve(j.req, 1) + kMargin;
        if (!fits(s, need, e)) return false;
        std::vector<uint64_t> members{*it};
        if (batchable(j)) {
            for (auto o = std::next(it); o != s->queue.end() && (int)members.size() < bm::kBatchMax; ++o) {
                const Job& oj = s->jobs[*o];
                if (!same_batch(j, oj)) continue;
                const int R = (int)members.size();
                const int64_t need2 = need - est_solve(j.req, R) + est_solve(j.req, R + 1);
                if (!fits(s, need2, e)) break;
                need = need2;
                members.push_back(*o);
            }
        }
        make_room(s, need, e, plan.victims);
        if (key && !e) {
            e = new Resident();
            e->key = key;
            e->npix = j.req.npix;
            e->nsamples = j.req.nsamples;
            e->solver = (int)j.req.solver;
            e->det_off = j.det_off;
            e->bytes = est_resident(j.req);
            s->resident[key] = e;
        }
        if (e) e->in_use = true;
        plan.entry = e;
        plan.resident_hit = ready;
        plan.bytes = need;
        plan.tickets = members;
        for (uint64_t t : members) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), t));
        return true;
    }
    return false;
}

// An unkeyed request: the whole solve on the slot's context, released after.
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
    ctx->ws_generation += 1;
    return st;
}

// A context whose scratch comes from the device's default pool: released
// per request (the budget accounts per request) into memory that the other
// slots and the next request reuse without mapping it again.
bm_status make_context(int device, cudaStream_t* stream, bm_context** ctx) {
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(stream, cudaStreamNonBlocking) != cudaSuccess) {
        *stream = nullptr;
        return BM_ERR_CUDA;
    }
    const bm_status st = bm_context_create(device, *stream, ctx);
    if (st == BM_OK && (*ctx)->ws_pool) {
        cudaMemPoolDestroy((*ctx)->ws_pool);
        (*ctx)->ws_pool = nullptr;
    }
    // no graph capture in the server's solves: a capture in a slot would make
    // a device-wide synchronisation by any other thread of the process fail
    if (st == BM_OK) (*ctx)->graphs = false;
    return st;
}

// Noise model and preconditioner of the entry for a request's settings.
bm_status build_noise(Resident* e, const Job& j) {
    bm_precond_destroy(e->pc);
    bm_inv_noise_destroy(e->n);
    e->pc = nullptr;
    e->n = nullptr;
    const bm_request& r = j.req;
    bm_status st;
    if (r.noise == BM_NOISE_WHITE)
        st = bm_inv_noise_create_diag(e->ctx, r.ndet, j.det_off.data(), j.inv_var.data(), &e->n);
    else
        st = bm_inv_noise_create_toeplitz(e->ctx, r.ndet, j.det_off.data(), r.chunk_len, r.nlags, j.coeffs.data(),
                                          j.inv_var.data(), &e->n);
    if (st == BM_OK) st = bm_blockdiag_precond_create(e->p, e->n, r.min_hits, r.max_cond, &e->pc);
    e->sig = st == BM_OK ? noise_sig(j) : NoiseSig{};
    return st;
}

bm_status build_entry(int device, Resident* e, const Job& j) {
    bm_status st = make_context(device, &e->stream, &e->ctx);
    const bm_request& r = j.req;
    if (st == BM_OK) {
        if (r.cos2psi)
            st = bm_pointing_create_trig(e->ctx, r.npix, r.nsamples, r.pix, r.cos2psi, r.sin2psi, r.solver, &e->p);
        else
            st = bm_pointing_create(e->ctx, r.npix, r.nsamples, r.pix, r.psi, r.psi_dtype, r.solver, &e->p);
    }
    if (st == BM_OK) st = build_noise(e, j);
    return st;
}

// The multi-RHS solve of a batch on the entry (white noise, mixed).
bm_status solve_batch(Resident* e, const std::vector<Job*>& js) {
    const int R = (int)js.size();
    std::vector<const void*> rows(R);
    std::vector<double*> maps(R);
    for (int r = 0; r < R; ++r) {
        rows[r] = js[r]->req.tod;
        maps[r] = js[r]->req.map_out;
    }
    std::vector<bm_solve_info> info(R);
    const bm_request& r0 = js[0]->req;
    bm_status st;
    bm::clear_error();
    try {
        BM_CUDA(cudaSetDevice(e->ctx->device));
        bm::tl_stream = e->ctx->stream;
        st = bm::batched_white_solve_rows(e->p, e->n, e->pc, rows.data(), r0.tod_dtype, R, maps.data(), r0.tol,
                                          r0.maxiter, info.data());
    } catch (const bm::Error& er) {
        st = er.status;
    } catch (const std::bad_alloc&) {
        bm::set_error("host allocation failed");
        st = BM_ERR_OOM;
    } catch (...) {
        bm::set_error("unexpected internal error");
        st = BM_ERR_CUDA;
    }
    const bool per_rhs = st == BM_OK || st == BM_ERR_NOT_CONVERGED || st == BM_ERR_BREAKDOWN;
    for (int r = 0; r < R; ++r) {
        bm_result& res = js[r]->res;
        res.status = per_rhs ? info[r].status : st;
        res.iterations = per_rhs ? info[r].iterations : 0;
        res.outer_iterations = per_rhs ? info[r].outer_iterations : 0;
        res.rel_residual = per_rhs ? info[r].rel_residual : 0.0;
    }
    return per_rhs ? BM_OK : st;
}

// A plan on its entry: build the entry (or its noise model) when needed,
// then one solve or the batch's multi-RHS solve.  Per-request statuses go
// to the jobs' results; the return value is a failure of the whole plan.
bm_status run_keyed(bm_server* s, Plan& plan, const std::vector<Job*>& js) {
    Resident* e = plan.entry;
    const Job& j0 = *js[0];
    bm_status st = BM_OK;
    if (!e->ready) st = build_entry(s->device, e, j0);
    else if (!(e->sig == noise_sig(j0))) st = build_noise(e, j0);
    if (st == BM_OK) {
        if (js.size() == 1) {
            const bm_request& r = j0.req;
            bm_solve_info info{};
            st = bm_pcg_solve(e->p, e->n, e->pc, r.tod, r.tod_dtype, 1, r.map_out, r.tol, r.maxiter, r.precision,
                              &info);
            js[0]->res.status = st;
            js[0]->res.iterations = info.iterations;
            js[0]->res.outer_iterations = info.outer_iterations;
            js[0]->res.rel_residual = info.rel_residual;
            if (st == BM_ERR_NOT_CONVERGED || st == BM_ERR_BREAKDOWN) st = BM_OK;  // the request's own status
        } else {
            st = solve_batch(e, js);
        }
    }
    if (e->ctx) {  // the solve's scratch goes back (the entry keeps its handles)
        cudaSetDevice(e->ctx->device);
        cudaStreamSynchronize(e->ctx->stream);
        e->ctx->ws.clear();
        e->ctx->ws_generation += 1;
    }
    return st;
}

}  // namespace

namespace {

void worker_main(bm_server* s, int slot) {
    cudaStream_t stream = nullptr;
    bm_context* ctx = nullptr;
    const bool ok = make_context(s->device, &stream, &ctx) == BM_OK;
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        Plan plan;
        s->cv_work.wait(lk, [&] { return s->stopping || pick(s, plan); });
        if (s->stopping) break;
        const auto t_start = Clock::now();
        std::vector<Job*> js;
        for (uint64_t t : plan.tickets) {
            Job& j = s->jobs[t];
            j.state = JobState::Running;
            j.t_start = t_start;
            j.res.slot = slot;
            js.push_back(&j);
        }
        s->reserved += plan.bytes;
        s->peak_reserved = std::max(s->peak_reserved, s->reserved);
        s->running += (int64_t)js.size();
        lk.unlock();

        for (Resident* v : plan.victims) destroy_resident(v);
        bm_status st;
        if (plan.reject) {
            bm::set_error("pointing_key %llu names a resident pointing of another shape (npix, nsamples, solver "
                          "or det_offsets)", (unsigned long long)js[0]->req.pointing_key);
            st = BM_ERR_INVALID;
        } else if (!ok) {
            st = BM_ERR_CUDA;
        } else if (plan.entry) {
            st = run_keyed(s, plan, js);
        } else {
            st = run_request(ctx, *js[0]);
            js[0]->res.status = st;
            if (st == BM_ERR_NOT_CONVERGED || st == BM_ERR_BREAKDOWN) st = BM_OK;
        }
        char msg[sizeof(bm_result::message)] = "";
        if (st != BM_OK) std::snprintf(msg, sizeof(msg), "%s", ok ? bm_last_error() : "worker context failed");
        else if (js[0]->res.status != BM_OK) std::snprintf(msg, sizeof(msg), "%s", bm_last_error());

        std::vector<Resident*> dead;
        lk.lock();
        Resident* e = plan.entry;
        if (e) {
            const bool built = e->p && e->n && e->pc;
            if (!e->ready && built && st == BM_OK) {
                e->ready = true;
                s->resident_total += e->bytes;
            }
            if (!e->ready) {  // the entry could not be built: drop it
                s->resident.erase(e->key);
                dead.push_back(e);
            } else {
                e->in_use = false;
                e->last_use = ++s->tick;
            }
        }
        s->reserved -= plan.bytes;
        s->running -= (int64_t)js.size();
        bool idle_entries = false;
        for (const auto& kv : s->resident) idle_entries = idle_entries || (kv.second->ready && !kv.second->in_use);
        if (st == BM_ERR_OOM && js[0]->oom_retries < kMaxOomRetries && (s->running > 0 || idle_entries)) {
            // Others hold memory: queue the requests again at the front, to
            // run after one of them completes; release the idle entries now.
            for (auto it = js.rbegin(); it != js.rend(); ++it) {
                Job& j = **it;
                j.state = JobState::Queued;
                j.oom_retries += 1;
                j.wait_completed = s->running > 0 ? s->completed : -1;
                j.res = bm_result{};
                s->queue.push_front(j.ticket);
            }
            s->oom_requeues += (int64_t)js.size();
            std::vector<Resident*> idle;
            for (auto it = s->resident.begin(); it != s->resident.end();) {
                Resident* r = it->second;
                if (r->ready && !r->in_use) {
                    s->resident_total -= r->bytes;
                    s->evictions += 1;
                    idle.push_back(r);
                    it = s->resident.erase(it);
                } else {
                    ++it;
                }
            }
            dead.insert(dead.end(), idle.begin(), idle.end());
        } else {
            const auto t_done = Clock::now();
            const int R = (int)js.size();
            for (Job* jp : js) {
                Job& j = *jp;
                j.t_done = t_done;
                if (st != BM_OK) j.res.status = st;
                std::memcpy(j.res.message, j.res.status == BM_OK ? "" : msg, sizeof(msg));
                j.res.queue_ms = ms_between(j.t_submit, j.t_start);
                j.res.run_ms = ms_between(j.t_start, j.t_done);
                j.res.latency_ms = ms_between(j.t_submit, j.t_done);
                j.res.device_bytes = plan.bytes / R;
                j.res.batch_size = R;
                j.res.resident = plan.resident_hit ? 1 : 0;
                j.state = JobState::Done;
                s->completed += 1;
                s->samples_done += (double)j.req.nsamples;
                s->latencies.push_back(j.res.latency_ms);
            }
            if (plan.resident_hit) s->resident_hits += R;
            if (R > 1) {
                s->batches += 1;
                s->batched_requests += R;
            }
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
        if (!dead.empty()) {
            lk.unlock();
            for (Resident* d : dead) destroy_resident(d);
            lk.lock();
        }
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
    job.bytes = est_resident(r) + est_create(r) + est_solve(r, 1) + kMargin;  // alone, nothing resident
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
    st.resident_bytes = s->resident_total;
    st.resident_hits = s->resident_hits;
    st.batches = s->batches;
    st.batched_requests = s->batched_requests;
    st.evictions = s->evictions;
    st.oom_requeues = s->oom_requeues;
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
    for (auto& kv : s->resident) destroy_resident(kv.second);
    s->resident.clear();
    // the slots' memory went back to the device's default pool, which keeps
    // it cached: hand it back to the device
    cudaMemPool_t pool = nullptr;
    if (cudaSetDevice(s->device) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
        cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess)
        cudaMemPoolTrimTo(pool, 0);
    delete s;
}

}  // extern "C"
